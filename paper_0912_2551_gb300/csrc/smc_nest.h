// smc_nest.h -- the trace monitor: BLTLc formulas of any nesting (Sec. 3.1)
// decided on the recorded prefix of a trajectory (the paper's lookahead
// buffer of Sec. 3.2, one per lane).  Host and device code, so that a host
// program can check it (tests/monitor_host.cpp).
//
// Knowledge points (the order in which the SSA learns about a path):
//   q = 2k      positions 0..k are known (entry times and states); the next
//               entry time is only known to be >= t_k;
//   q = 2k + 1  positions 0..k are known and the entry time of position
//               k + 1 has been drawn (or the path absorbed after k, or, for
//               a replayed prefix, a lower bound of it is given).
// Knowledge only grows with q, so a subformula's three-valued value at a
// position, once true or false, stays so.  nest_eval returns, for a node at
// position j, that value and the first knowledge point at which it holds
// (the decision point); the formula's verdict and the point at which the
// trajectory stops (Sec. 3.2: as soon as the verdict is fixed) are those of
// the root at position 0.
//
// Until (phi U[a,b] psi at j, Sec. 3.1: some m with t_m - t_j in [a,b],
// psi at m and phi at every j <= p < m) is decided
//   true  at the first q by which some such witness m has psi and every phi
//         before it known true: min over m of max(D_psi(m), D_phi(p < m));
//   false at the first q by which the scan of the positions in order (psi
//         at a candidate m considered before phi at m) ends -- at a position
//         where phi is known false, or where the window is known to have
//         closed -- with psi known false at every candidate up to there.
// F[a,b] psi = tt U[a,b] psi; G[a,b] psi = not F[a,b] not psi; X[a,b] psi at
// j: position j + 1 is entered after a sojourn in [a, b] and satisfies psi.
// The evaluation recurses on the formula tree (depth bounded at compile
// time: no run-time recursion).  Without a memo it rescans windows, so its
// cost grows with the product of the nested windows' lengths in positions.
// With one (NestTrace::memo), every temporal node below another temporal
// node keeps, per position, its value once decided -- final, since
// knowledge only grows -- or the knowledge point at which it was last found
// undetermined; each such value is then computed once per knowledge point
// at most, and a decided one once per path.
#pragma once
#include <stdint.h>

#include "smc.h"

#ifdef __CUDACC__
#define SMC_NEST_HD __host__ __device__
#else
#define SMC_NEST_HD
#endif
#if defined(__CUDA_ARCH__)
#define SMC_NEST_NOINLINE __noinline__
#define SMC_NEST_SUB(x, y) __dsub_rn((x), (y))
#define SMC_NEST_ADD(x, y) __dadd_rn((x), (y))
#else
#include <string.h>
#define SMC_NEST_NOINLINE
#define SMC_NEST_SUB(x, y) ((x) - (y))
#define SMC_NEST_ADD(x, y) ((x) + (y))
#endif

#define SMC_NEST_MAX_NODES 32
#define SMC_NEST_MAX_DEPTH 10  // height of the formula tree (nodes on a root-leaf path)

// Node kinds are the SMC_NODE_* codes of smc.h; c0, c1 operands (c0 the
// left one of Until), bit the atom's bit in the state's atom vector, [lo, hi]
// the interval of a temporal operator.
// slot: the node's memo column (a temporal node with a temporal ancestor),
// else -1.
struct NestNode {
    int32_t kind, c0, c1, bit;
    int32_t slot, pad_;
    double lo, hi;
};

struct NestProg {
    int32_t n_nodes, root, height;
    int32_t unbounded;  // the formula's horizon is infinite: pessimistic rule at t_stop
    int32_t n_slots;    // memo columns (nodes with slot >= 0)
    int32_t pad_;
    double t_static;    // latest time at which a position can still matter (+inf: unbounded)
    double t_stop;      // t_static, or t_max_unbounded for an unbounded formula
    NestNode nd[SMC_NEST_MAX_NODES];
};

// What is known of a path: positions 0..E (entry times t[m * s], atom bit
// vectors w[m * s] in bits 0-23; s the stride between positions, 1 for a
// contiguous recording) and, after position E, `end`:
//   0  nothing (the last knowledge point is 2E);
//   1  the entry time tnext of position E + 1, drawn (2E + 1);
//   2  the path absorbed after E, no further position (2E + 1);
//   3  a lower bound tnext of the next entry time (2E + 1; replay only).
// memo (optional): slot k's cell for position m at memo[k * mslot + m * s];
// 0 unknown, else (d << 2) | v for a decided value (v = 1 false, 2 true),
// (q << 2) | 3 for one undetermined at knowledge point q.  Whoever records
// position m zeroes its cells first; the knowledge points at which one
// memo is used must not decrease (the SSA's order: memo values of a
// trajectory are final or tied to the point that computed them).
struct NestTrace {
    const double *t;
    const uint32_t *w;
    int64_t s;
    int64_t E;
    int32_t end;
    double tnext;
    uint32_t *memo;
    int64_t mslot;
};

// v: 0 undetermined, 1 false, 2 true (the monitor's codes); d: the decision
// point, kNestNever while undetermined
struct NestVal {
    int32_t v;
    int64_t d;
};
#define SMC_NEST_NEVER ((int64_t)0x7FFFFFFFFFFFFFFFll)

SMC_NEST_HD inline int nest_not(int v) { return v == 0 ? 0 : 3 - v; }
SMC_NEST_HD inline int64_t nest_min(int64_t a, int64_t b) { return a < b ? a : b; }
SMC_NEST_HD inline int64_t nest_max(int64_t a, int64_t b) { return a > b ? a : b; }

// Kleene and / or of two decided-at values: false (true) as soon as one
// operand is, true (false) once both are
SMC_NEST_HD inline NestVal nest_and(NestVal a, NestVal b)
{
    if (a.v == 1 && b.v == 1) return {1, nest_min(a.d, b.d)};
    if (a.v == 1) return a;
    if (b.v == 1) return b;
    if (a.v == 2 && b.v == 2) return {2, nest_max(a.d, b.d)};
    return {0, SMC_NEST_NEVER};
}

SMC_NEST_HD inline NestVal nest_or(NestVal a, NestVal b)
{
    if (a.v == 2 && b.v == 2) return {2, nest_min(a.d, b.d)};
    if (a.v == 2) return a;
    if (b.v == 2) return b;
    if (a.v == 1 && b.v == 1) return {1, nest_max(a.d, b.d)};
    return {0, SMC_NEST_NEVER};
}

SMC_NEST_HD inline int64_t nest_bits(double x)
{
#if defined(__CUDA_ARCH__)
    return __double_as_longlong(x);
#else
    int64_t b;
    memcpy(&b, &x, 8);
    return b;
#endif
}

SMC_NEST_HD inline double nest_from_bits(int64_t b)
{
#if defined(__CUDA_ARCH__)
    return __longlong_as_double(b);
#else
    double x;
    memcpy(&x, &b, 8);
    return x;
#endif
}

// The window tests of the scans (t - t_j > b, t - t_j >= a, rounded as the
// oracle rounds them) on the integer pipes.  Rounded subtraction is
// monotone in its first operand, so over times t >= 0 each test holds on an
// interval of t, and bit patterns of non-negative doubles order like their
// values: t - t_j <= b iff bits(t) <= nest_last_within(t_j, b), and
// t - t_j >= a iff bits(t) >= nest_first_reaching(t_j, a).  The boundary
// lies within an ulp or two of the rounded t_j + b (t_j + a); it is
// searched for there and confirmed (it passes, its neighbour fails).
// -1 when the confirmation fails (bounds near the top of the double
// range): the scan then subtracts.
SMC_NEST_HD inline int64_t nest_last_within(double tj, double b)
{
    const int64_t inf = 0x7FF0000000000000ll;
    if (!(b < nest_from_bits(inf))) return inf;  // b = +inf: every time lies within
    int64_t xb = nest_bits(SMC_NEST_ADD(tj, b));
    auto within = [&](int64_t x) { return SMC_NEST_SUB(nest_from_bits(x), tj) <= b; };
    for (int k = 0; k < 4 && xb > 0 && !within(xb); ++k) --xb;
    for (int k = 0; k < 4 && xb < inf && within(xb + 1); ++k) ++xb;
    return (xb >= 0 && xb < inf && within(xb) && !within(xb + 1)) ? xb : -1;
}

SMC_NEST_HD inline int64_t nest_first_reaching(double tj, double a)
{
    const int64_t inf = 0x7FF0000000000000ll;
    int64_t xb = nest_bits(SMC_NEST_ADD(tj, a));
    auto reach = [&](int64_t x) { return SMC_NEST_SUB(nest_from_bits(x), tj) >= a; };
    for (int k = 0; k < 4 && xb < inf && !reach(xb); ++k) ++xb;
    for (int k = 0; k < 4 && xb > 0 && reach(xb - 1); ++k) --xb;
    return (xb >= 0 && xb <= inf && reach(xb) && (xb == 0 || !reach(xb - 1))) ? xb : -1;
}

template <int DEPTH>
SMC_NEST_HD SMC_NEST_NOINLINE NestVal nest_eval(const NestProg &P, const NestTrace &T, int node, int64_t j);

// A memo cell's value at knowledge point q: decided (final), undetermined
// at q, or not known (v = -1: the node must be evaluated).
SMC_NEST_HD inline NestVal nest_cell(uint32_t c, uint32_t q)
{
    if ((c & 3u) == 1u || (c & 3u) == 2u) return {(int32_t)(c & 3u), (int64_t)(c >> 2)};
    if (c == ((q << 2) | 3u)) return {0, SMC_NEST_NEVER};
    return {-1, 0};
}

// A node's value at position j: atoms and memo hits in line, the rest by
// the (out-of-line) evaluator
template <int DEPTH>
SMC_NEST_HD inline NestVal nest_child(const NestProg &P, const NestTrace &T, int node, int64_t j)
{
    const NestNode &n = P.nd[node];
    if (n.kind == SMC_NODE_ATOM) return {((T.w[j * T.s] >> n.bit) & 1u) ? 2 : 1, 2 * j};
    if (T.memo && n.slot >= 0) {
        const NestVal c = nest_cell(T.memo[n.slot * T.mslot + j * T.s], (uint32_t)(2 * T.E + (T.end != 0)));
        if (c.v >= 0) return c;
    }
    return nest_eval<DEPTH>(P, T, node, j);
}

// phi U[a,b] psi at position j (l = -1: phi = tt; neg: psi negated, for G)
template <int DEPTH>
SMC_NEST_HD SMC_NEST_NOINLINE NestVal nest_until(const NestProg &P, const NestTrace &T, int l, int r, bool neg,
                                                 double a, double b, int64_t j)
{
    int64_t dT = SMC_NEST_NEVER, dF = SMC_NEST_NEVER;
    bool canT = true, canF = true;  // a later witness / a later end can still decide
    int64_t maxDl = 0, maxDr = 0;   // phi known true on [j, m); psi known false at the candidates so far
    bool stopped = false;
    const double tj = T.t[j * T.s];
    const int64_t last_in = nest_last_within(tj, b), first_in = nest_first_reaching(tj, a);
    auto beyond = [&](double t) { return last_in >= 0 ? nest_bits(t) > last_in : SMC_NEST_SUB(t, tj) > b; };
    for (int64_t m = j; m <= T.E; ++m) {
        const double tm = T.t[m * T.s];
        if (beyond(tm)) {  // the window is known closed once position m's entry time is drawn
            if (canF) dF = nest_min(dF, nest_max(2 * m - 1, maxDr));
            stopped = true;
            break;
        }
        if (first_in >= 0 ? nest_bits(tm) >= first_in : SMC_NEST_SUB(tm, tj) >= a) {  // candidate witness
            NestVal rv = nest_child<DEPTH - 1>(P, T, r, m);
            if (neg) rv.v = nest_not(rv.v);
            if (canT && rv.v == 2) dT = nest_min(dT, nest_max(rv.d, maxDl));
            if (rv.v != 1) canF = false;
            else maxDr = nest_max(maxDr, rv.d);
        }
        if (l >= 0) {
            const NestVal lv = nest_child<DEPTH - 1>(P, T, l, m);
            if (lv.v == 1 && canF) dF = nest_min(dF, nest_max(lv.d, maxDr));  // the scan ends here
            if (lv.v != 2) canT = false;
            else maxDl = nest_max(maxDl, lv.d);
        }
        // nothing later decides earlier: later candidates and ends are known
        // at 2(m + 1) - 1 or after
        if ((!canT && !canF) || nest_min(dT, dF) <= 2 * m + 1) {
            stopped = true;
            break;
        }
    }
    if (!stopped && canF) {  // every position scanned: the window closes after E, or never here
        const bool shut = T.end == 2 || ((T.end == 1 || T.end == 3) && beyond(T.tnext));
        if (shut) dF = nest_min(dF, nest_max(2 * T.E + 1, maxDr));
    }
    if (dT != SMC_NEST_NEVER && dT <= dF) return {2, dT};
    if (dF != SMC_NEST_NEVER) return {1, dF};
    return {0, SMC_NEST_NEVER};
}

template <>
SMC_NEST_HD inline NestVal nest_eval<0>(const NestProg &, const NestTrace &, int, int64_t)
{
    return {0, SMC_NEST_NEVER};  // deeper than SMC_NEST_MAX_DEPTH: the compiler rejects such formulas
}

template <int DEPTH>
SMC_NEST_HD SMC_NEST_NOINLINE NestVal nest_eval(const NestProg &P, const NestTrace &T, int node, int64_t j)
{
    const NestNode &n = P.nd[node];
    switch (n.kind) {
    case SMC_NODE_TRUE: return {2, 2 * j};
    case SMC_NODE_FALSE: return {1, 2 * j};
    case SMC_NODE_ATOM: return {((T.w[j * T.s] >> n.bit) & 1u) ? 2 : 1, 2 * j};
    case SMC_NODE_NOT: {
        NestVal a = nest_child<DEPTH - 1>(P, T, n.c0, j);
        a.v = nest_not(a.v);
        return a;
    }
    case SMC_NODE_AND:
    case SMC_NODE_OR:
    case SMC_NODE_IMPLIES: {
        NestVal a = nest_child<DEPTH - 1>(P, T, n.c0, j);
        if (n.kind == SMC_NODE_IMPLIES) a.v = nest_not(a.v);
        // a first operand that settles the result at 2j (the earliest point a
        // value at position j can be known) leaves nothing for the second
        if (a.d == 2 * j && a.v == (n.kind == SMC_NODE_AND ? 1 : 2)) return a;
        const NestVal b = nest_child<DEPTH - 1>(P, T, n.c1, j);
        return n.kind == SMC_NODE_AND ? nest_and(a, b) : nest_or(a, b);
    }
    case SMC_NODE_UNTIL:
    case SMC_NODE_EVENTUALLY:
    case SMC_NODE_ALWAYS: {
        const uint32_t q = (uint32_t)(2 * T.E + (T.end != 0));  // this knowledge point
        uint32_t *cell = nullptr;
        if (T.memo && n.slot >= 0) {
            cell = T.memo + n.slot * T.mslot + j * T.s;
            const NestVal c = nest_cell(*cell, q);
            if (c.v >= 0) return c;
        }
        NestVal g = n.kind == SMC_NODE_UNTIL
                        ? nest_until<DEPTH>(P, T, n.c0, n.c1, false, n.lo, n.hi, j)
                        : nest_until<DEPTH>(P, T, -1, n.c0, n.kind == SMC_NODE_ALWAYS, n.lo, n.hi, j);
        if (n.kind == SMC_NODE_ALWAYS) g.v = nest_not(g.v);
        if (cell) *cell = g.v ? (((uint32_t)g.d << 2) | (uint32_t)g.v) : ((q << 2) | 3u);
        return g;
    }
    case SMC_NODE_NEXT: {
        if (j < T.E) {  // position j + 1 is known; its entry time was drawn at 2j + 1
            const double d = SMC_NEST_SUB(T.t[(j + 1) * T.s], T.t[j * T.s]);
            if (d < n.lo || d > n.hi) return {1, 2 * j + 1};
            return nest_child<DEPTH - 1>(P, T, n.c0, j + 1);
        }
        if (T.end == 2) return {1, 2 * j + 1};  // no next position
        if (T.end == 1 || T.end == 3) {
            const double d = SMC_NEST_SUB(T.tnext, T.t[j * T.s]);
            if (d > n.hi || (T.end == 1 && d < n.lo)) return {1, 2 * j + 1};
        }
        return {0, SMC_NEST_NEVER};
    }
    default: return {0, SMC_NEST_NEVER};
    }
}

// The formula at position 0: its verdict and the knowledge point fixing it.
SMC_NEST_HD inline NestVal nest_decide(const NestProg &P, const NestTrace &T)
{
    return nest_eval<SMC_NEST_MAX_DEPTH>(P, T, P.root, 0);
}
