// Host check of the formula compiler and atom helpers of
// paper_0912_2551_gb300/csrc/smc_compile.cpp (host code of the library):
//  * atom_threshold: an atom L <op> b over integer L becomes lo <= L <= hi
//    (negated for !=); checked by brute force against the FP64 comparison
//    (double)L <op> b for every operator, integer and fractional bounds,
//    ties, and bounds beyond the saturation limit;
//  * validate_tokens: accepted and rejected postfix atom programs;
//  * parse_formula: well-formed and malformed postfix formulas;
//  * compile_formula: the monitor units of the workloads' formulas (windows,
//    left / right / nested truth tables over the atom bit vector) and the
//    three-valued verdict table of boolean combinations of temporal
//    operators, checked against Kleene's strong three-valued logic; and
//    every formula outside the monitorable fragment is rejected;
//  * compile_nested (the trace monitor's program): those rejected shapes
//    compile; horizons (each temporal operator adds its interval end to its
//    operands'), memo columns exactly on the U / F / G nodes below another
//    temporal operator, tree height 10 / 32 nodes / 6 atoms accepted and
//    one more rejected, bad intervals, unbounded formulas and t_max.
// Prints "ok" and exits 0 when every check holds.
#include <math.h>
#include <stdint.h>
#include <stdio.h>

#include <functional>
#include <limits>
#include <string>
#include <vector>

#include "smc.h"
#include "smc_compile.h"

using namespace smc;

static int failures = 0;
#define CHECK(c)                                                                 \
    do {                                                                         \
        if (!(c)) {                                                              \
            ++failures;                                                          \
            if (failures < 30) printf("FAIL line %d: %s\n", __LINE__, #c);       \
        }                                                                        \
    } while (0)

// ---------------------------------------------------------------- atoms
static bool fp64_compare(int op, double l, double b)
{
    switch (op) {
    case SMC_OP_LT: return l < b;
    case SMC_OP_LE: return l <= b;
    case SMC_OP_GE: return l >= b;
    case SMC_OP_GT: return l > b;
    case SMC_OP_EQ: return l == b;
    case SMC_OP_NE: return l != b;
    }
    return false;
}

static void check_thresholds()
{
    const double bounds[] = {0.0, -0.0, 1.0, -1.0, 7.0, -7.0, 0.5, -0.5, 2.25, -2.25, 130.0, 129.999999, 130.000001,
                             1e-300, -1e-300, 1e6, -1e6, 3.5e15, 5e18, -5e18, 1e300, -1e300, 4.0e18, -4.0e18};
    long checked = 0;
    for (int op = SMC_OP_LT; op <= SMC_OP_NE; ++op)
        for (double b : bounds) {
            int64_t lo, hi;
            bool neg;
            atom_threshold(op, b, lo, hi, neg);
            auto holds = [&](int64_t L) { return (lo <= L && L <= hi) != neg; };
            for (int64_t L = -300; L <= 300; ++L) {
                CHECK(holds(L) == fp64_compare(op, (double)L, b));
                ++checked;
            }
            // around the bound itself and far out (|L| < 2^53: exact doubles)
            if (fabs(b) < 1e15) {
                const int64_t c = (int64_t)floor(b);
                for (int64_t L = c - 3; L <= c + 3; ++L) CHECK(holds(L) == fp64_compare(op, (double)L, b));
            }
            for (int64_t L : {(int64_t)1 << 52, -((int64_t)1 << 52), (int64_t)4000000000000000LL})
                CHECK(holds(L) == fp64_compare(op, (double)L, b));
        }
    CHECK(checked > 80000);
}

// ---------------------------------------------------------------- tokens
static smc_token tk(int kind, int arg = 0, double v = 0.0)
{
    smc_token t;
    t.kind = kind;
    t.arg = arg;
    t.value = v;
    return t;
}

static void check_tokens()
{
    std::string err;
    const int S = 3;
    // x0 / sqrt(x1 + 2)  and  x2^3 - 1
    const std::vector<smc_token> good1 = {tk(SMC_TOK_SPECIES, 0), tk(SMC_TOK_SPECIES, 1), tk(SMC_TOK_CONST, 0, 2.0),
                                          tk(SMC_TOK_ADD), tk(SMC_TOK_SQRT), tk(SMC_TOK_DIV)};
    const std::vector<smc_token> good2 = {tk(SMC_TOK_SPECIES, 2), tk(SMC_TOK_POWI, 3), tk(SMC_TOK_CONST, 0, 1.0),
                                          tk(SMC_TOK_SUB)};
    CHECK(validate_tokens(good1.data(), (int)good1.size(), S, err) == SMC_OK);
    CHECK(validate_tokens(good2.data(), (int)good2.size(), S, err) == SMC_OK);
    const int32_t x[3] = {14, 47, 2};
    CHECK(eval_tokens(good1.data(), (int)good1.size(), x) == 14.0 / sqrt(49.0));
    CHECK(eval_tokens(good2.data(), (int)good2.size(), x) == 7.0);
    const std::vector<std::vector<smc_token>> bad = {
        {},                                                                   // empty
        {tk(SMC_TOK_SPECIES, 3)},                                             // species out of range
        {tk(SMC_TOK_SPECIES, -1)},
        {tk(SMC_TOK_CONST, 0, INFINITY)},                                     // non-finite constant
        {tk(SMC_TOK_CONST, 0, NAN)},
        {tk(SMC_TOK_SPECIES, 0), tk(SMC_TOK_ADD)},                            // operator with one operand
        {tk(SMC_TOK_SQRT)},                                                   // sqrt of nothing
        {tk(SMC_TOK_SPECIES, 0), tk(SMC_TOK_POWI, 17)},                       // power beyond 16
        {tk(SMC_TOK_SPECIES, 0), tk(SMC_TOK_POWI, -1)},
        {tk(SMC_TOK_SPECIES, 0), tk(SMC_TOK_SPECIES, 1)},                     // two values left
        {tk(99)},                                                             // unknown token
    };
    for (const auto &b : bad) CHECK(validate_tokens(b.data(), (int)b.size(), S, err) == SMC_E_INVALID_ARG);
    std::vector<smc_token> deep;
    for (int i = 0; i < 9; ++i) deep.push_back(tk(SMC_TOK_CONST, 0, 1.0));  // stack of 9 > 8
    for (int i = 0; i < 8; ++i) deep.push_back(tk(SMC_TOK_ADD));
    CHECK(validate_tokens(deep.data(), (int)deep.size(), S, err) == SMC_E_INVALID_ARG);
    std::vector<smc_token> longp;
    longp.push_back(tk(SMC_TOK_CONST, 0, 1.0));
    for (int i = 0; i < 16; ++i) { longp.push_back(tk(SMC_TOK_CONST, 0, 1.0)); longp.push_back(tk(SMC_TOK_ADD)); }
    CHECK((int)longp.size() == 33 && validate_tokens(longp.data(), 33, S, err) == SMC_E_INVALID_ARG);
    longp.resize(31);  // 31 tokens, depth 2: accepted
    CHECK(validate_tokens(longp.data(), 31, S, err) == SMC_OK);
}

// ---------------------------------------------------------------- formulas
static smc_node nd(int kind, int arg = 0, double lo = 0.0, double hi = 0.0)
{
    smc_node n;
    n.kind = kind;
    n.arg = arg;
    n.lo = lo;
    n.hi = hi;
    return n;
}

static int compile(const std::vector<smc_node> &f, int n_atoms, double t_max, MonProg &prog, std::string &err)
{
    std::vector<FNode> tree;
    int root = -1;
    int rc = parse_formula(f.data(), (int)f.size(), n_atoms, tree, root, err);
    if (rc != SMC_OK) return rc;
    std::vector<int> used;
    return compile_formula(tree, root, n_atoms, t_max, prog, used, err);
}

// truth table over the 6-bit atom vector of a predicate on the bits
template <class F>
static uint64_t table(F f)
{
    uint64_t t = 0;
    for (uint32_t b = 0; b < 64; ++b)
        if (f(b)) t |= 1ull << b;
    return t;
}

enum { U = 0, FF = 1, TT = 2 };  // undetermined, false, true
static int k_not(int a) { return a == U ? U : (a == TT ? FF : TT); }
static int k_and(int a, int b) { return (a == FF || b == FF) ? FF : (a == TT && b == TT) ? TT : U; }
static int k_or(int a, int b) { return k_not(k_and(k_not(a), k_not(b))); }

static void check_formulas()
{
    std::string err;
    MonProg p;
    const double inf = std::numeric_limits<double>::infinity();
    const auto A0 = [](uint32_t b) { return (b & 1u) != 0; };
    const auto A1 = [](uint32_t b) { return (b & 2u) != 0; };
    const auto A2 = [](uint32_t b) { return (b & 4u) != 0; };

    // F[0,100] (A >= 130)
    CHECK(compile({nd(SMC_NODE_ATOM, 0), nd(SMC_NODE_EVENTUALLY, 0, 0.0, 100.0)}, 1, inf, p, err) == SMC_OK);
    CHECK(p.n_units == 1 && p.n_atoms == 1 && p.u[0].nest == 0 && p.u[0].a == 0.0 && p.u[0].b == 100.0);
    CHECK(p.u[0].L == ~0ull && p.u[0].P == table(A0) && !p.unbounded && !p.has_lower);
    CHECK(p.table[U] == U && p.table[FF] == FF && p.table[TT] == TT);

    // G[0,30] (X > 0 & Y > 0) = not F[0,30] not (...)
    CHECK(compile({nd(SMC_NODE_ATOM, 0), nd(SMC_NODE_ATOM, 1), nd(SMC_NODE_AND), nd(SMC_NODE_ALWAYS, 0, 0.0, 30.0)}, 2,
                  inf, p, err) == SMC_OK);
    CHECK(p.n_units == 1 && p.u[0].b == 30.0 && p.u[0].P == table([&](uint32_t b) { return !(A0(b) && A1(b)); }));
    CHECK(p.table[U] == U && p.table[FF] == TT && p.table[TT] == FF);

    // (KPP < 500) U[0,200] (KPP >= 2000 & F[0,50] KPP < 500)
    CHECK(compile({nd(SMC_NODE_ATOM, 0), nd(SMC_NODE_ATOM, 1), nd(SMC_NODE_ATOM, 2),
                   nd(SMC_NODE_EVENTUALLY, 0, 0.0, 50.0), nd(SMC_NODE_AND), nd(SMC_NODE_UNTIL, 0, 0.0, 200.0)},
                  3, inf, p, err) == SMC_OK);
    CHECK(p.n_units == 1 && p.u[0].nest == 1 && p.u[0].d == 50.0 && p.u[0].b == 200.0);
    CHECK(p.u[0].L == table(A0) && p.u[0].P == table(A1) && p.u[0].Q == table(A2));

    // a nested G: F[0,10] (A1 & G[0,5] A2)
    CHECK(compile({nd(SMC_NODE_ATOM, 1), nd(SMC_NODE_ATOM, 2), nd(SMC_NODE_ALWAYS, 0, 0.0, 5.0), nd(SMC_NODE_AND),
                   nd(SMC_NODE_EVENTUALLY, 0, 0.0, 10.0)},
                  3, inf, p, err) == SMC_OK);
    CHECK(p.n_units == 1 && p.u[0].nest == 2 && p.u[0].d == 5.0);
    CHECK(p.u[0].P == table([](uint32_t b) { return (b & 1u) != 0; }) && p.u[0].Q == table([](uint32_t b) { return (b & 2u) != 0; }));

    // X[0.05, 0.2] (A >= 1)
    CHECK(compile({nd(SMC_NODE_ATOM, 0), nd(SMC_NODE_NEXT, 0, 0.05, 0.2)}, 1, inf, p, err) == SMC_OK);
    CHECK(p.n_units == 1 && p.u[0].nest == 3 && p.u[0].a == 0.05 && p.u[0].b == 0.2 && p.u[0].P == table(A0));

    // boolean combinations: the table is Kleene logic over the units' values
    // (F[0,1] a0 & G[0,2] a1) | !(a2 U[1,3] a0)
    CHECK(compile({nd(SMC_NODE_ATOM, 0), nd(SMC_NODE_EVENTUALLY, 0, 0.0, 1.0), nd(SMC_NODE_ATOM, 1),
                   nd(SMC_NODE_ALWAYS, 0, 0.0, 2.0), nd(SMC_NODE_AND), nd(SMC_NODE_ATOM, 2), nd(SMC_NODE_ATOM, 0),
                   nd(SMC_NODE_UNTIL, 0, 1.0, 3.0), nd(SMC_NODE_NOT), nd(SMC_NODE_OR)},
                  3, inf, p, err) == SMC_OK);
    CHECK(p.n_units == 3 && p.has_lower);
    for (int v0 = 0; v0 < 3; ++v0)
        for (int v1 = 0; v1 < 3; ++v1)
            for (int v2 = 0; v2 < 3; ++v2) {
                // unit 1 is the F-form of G[0,2] a1: its value is that of F[0,2] !a1
                const int want = k_or(k_and(v0, k_not(v1)), k_not(v2));
                CHECK(p.table[v0 + 3 * v1 + 9 * v2] == want);
            }
    // implication: F[0,1] a0 -> G[0,1] a1
    CHECK(compile({nd(SMC_NODE_ATOM, 0), nd(SMC_NODE_EVENTUALLY, 0, 0.0, 1.0), nd(SMC_NODE_ATOM, 1),
                   nd(SMC_NODE_ALWAYS, 0, 0.0, 1.0), nd(SMC_NODE_IMPLIES)},
                  2, inf, p, err) == SMC_OK);
    CHECK(p.n_units == 2);
    for (int v0 = 0; v0 < 3; ++v0)
        for (int v1 = 0; v1 < 3; ++v1) CHECK(p.table[v0 + 3 * v1] == k_or(k_not(v0), k_not(v1)));

    // unbounded windows need t_max (the pessimistic rule)
    const std::vector<smc_node> unb = {nd(SMC_NODE_ATOM, 0), nd(SMC_NODE_EVENTUALLY, 0, 0.0, inf)};
    CHECK(compile(unb, 1, inf, p, err) == SMC_E_INVALID_ARG);
    CHECK(compile(unb, 1, 0.0, p, err) == SMC_E_INVALID_ARG);
    CHECK(compile(unb, 1, 10.0, p, err) == SMC_OK && p.unbounded && p.t_max == 10.0);

    // malformed postfix
    CHECK(compile({}, 1, inf, p, err) == SMC_E_INVALID_ARG);
    CHECK(compile({nd(SMC_NODE_AND)}, 1, inf, p, err) == SMC_E_INVALID_ARG);
    CHECK(compile({nd(SMC_NODE_ATOM, 0), nd(SMC_NODE_ATOM, 0)}, 1, inf, p, err) == SMC_E_INVALID_ARG);
    CHECK(compile({nd(SMC_NODE_ATOM, 1)}, 1, inf, p, err) == SMC_E_INVALID_ARG);
    CHECK(compile({nd(SMC_NODE_ATOM, -1)}, 1, inf, p, err) == SMC_E_INVALID_ARG);
    CHECK(compile({nd(42)}, 1, inf, p, err) == SMC_E_INVALID_ARG);

    // outside the monitorable fragment
    std::vector<smc_node> five;  // five temporal operators
    for (int i = 0; i < 5; ++i) {
        five.push_back(nd(SMC_NODE_ATOM, 0));
        five.push_back(nd(SMC_NODE_EVENTUALLY, 0, 0.0, 1.0 + i));
        if (i) five.push_back(nd(SMC_NODE_AND));
    }
    CHECK(compile(five, 1, inf, p, err) == SMC_E_UNSUPPORTED);
    five.resize(five.size() - 3);  // four: accepted
    CHECK(compile(five, 1, inf, p, err) == SMC_OK && p.n_units == 4);
    std::vector<smc_node> seven;  // seven distinct atoms
    for (int i = 0; i < 7; ++i) {
        seven.push_back(nd(SMC_NODE_ATOM, i));
        if (i) seven.push_back(nd(SMC_NODE_AND));
    }
    seven.push_back(nd(SMC_NODE_EVENTUALLY, 0, 0.0, 1.0));
    CHECK(compile(seven, 7, inf, p, err) == SMC_E_UNSUPPORTED);
    // X over a temporal operand; U with a temporal left operand; a nested
    // window not starting at 0; two nested operators in one operand
    CHECK(compile({nd(SMC_NODE_ATOM, 0), nd(SMC_NODE_EVENTUALLY, 0, 0.0, 1.0), nd(SMC_NODE_NEXT, 0, 0.0, 1.0)}, 1, inf,
                  p, err) == SMC_E_UNSUPPORTED);
    CHECK(compile({nd(SMC_NODE_ATOM, 0), nd(SMC_NODE_EVENTUALLY, 0, 0.0, 1.0), nd(SMC_NODE_ATOM, 1),
                   nd(SMC_NODE_UNTIL, 0, 0.0, 2.0)},
                  2, inf, p, err) == SMC_E_UNSUPPORTED);
    CHECK(compile({nd(SMC_NODE_ATOM, 0), nd(SMC_NODE_EVENTUALLY, 0, 1.0, 2.0), nd(SMC_NODE_EVENTUALLY, 0, 0.0, 5.0)}, 1,
                  inf, p, err) == SMC_E_UNSUPPORTED);
    CHECK(compile({nd(SMC_NODE_ATOM, 0), nd(SMC_NODE_EVENTUALLY, 0, 0.0, 1.0), nd(SMC_NODE_ATOM, 1),
                   nd(SMC_NODE_ALWAYS, 0, 0.0, 1.0), nd(SMC_NODE_AND), nd(SMC_NODE_EVENTUALLY, 0, 0.0, 5.0)},
                  2, inf, p, err) == SMC_E_UNSUPPORTED);
    // a nested F under a nested F (depth 3)
    CHECK(compile({nd(SMC_NODE_ATOM, 0), nd(SMC_NODE_EVENTUALLY, 0, 0.0, 1.0), nd(SMC_NODE_EVENTUALLY, 0, 0.0, 2.0),
                   nd(SMC_NODE_EVENTUALLY, 0, 0.0, 3.0)},
                  1, inf, p, err) == SMC_E_UNSUPPORTED);
    // windows must satisfy 0 <= lo <= hi
    CHECK(compile({nd(SMC_NODE_ATOM, 0), nd(SMC_NODE_EVENTUALLY, 0, 2.0, 1.0)}, 1, inf, p, err) != SMC_OK);
    CHECK(compile({nd(SMC_NODE_ATOM, 0), nd(SMC_NODE_EVENTUALLY, 0, -1.0, 1.0)}, 1, inf, p, err) != SMC_OK);
    CHECK(compile({nd(SMC_NODE_ATOM, 0), nd(SMC_NODE_EVENTUALLY, 0, 0.0, NAN)}, 1, inf, p, err) != SMC_OK);
}

// ---------------------------------------------------------------- trace monitor
static int compile_n(const std::vector<smc_node> &f, int n_atoms, double t_max, NestProg &np, std::string &err)
{
    std::vector<FNode> tree;
    int root = -1;
    int rc = parse_formula(f.data(), (int)f.size(), n_atoms, tree, root, err);
    if (rc != SMC_OK) return rc;
    std::vector<int> used;
    return compile_nested(tree, root, n_atoms, t_max, np, used, err);
}

static bool is_temporal(int k)
{
    return k == SMC_NODE_UNTIL || k == SMC_NODE_EVENTUALLY || k == SMC_NODE_ALWAYS || k == SMC_NODE_NEXT;
}

// Memo columns: exactly the U / F / G nodes with a temporal ancestor, numbered
// 0..n_slots-1 (an ancestor is found by walking down from the root).
static bool slots_ok(const NestProg &np)
{
    std::vector<int> under(np.n_nodes, 0), seen(np.n_slots, 0);
    std::vector<int> stack{np.root};
    while (!stack.empty()) {
        const int k = stack.back();
        stack.pop_back();
        const NestNode &n = np.nd[k];
        const bool want = under[k] && is_temporal(n.kind) && n.kind != SMC_NODE_NEXT;
        if (want != (n.slot >= 0)) return false;
        if (n.slot >= 0) {
            if (n.slot >= np.n_slots || seen[n.slot]) return false;
            seen[n.slot] = 1;
        }
        for (int c : {n.c0, n.c1})
            if (c >= 0) {
                under[c] = under[k] || is_temporal(n.kind);
                stack.push_back(c);
            }
    }
    for (int v : seen)
        if (!v) return false;
    return true;
}

static void check_nested()
{
    std::string err;
    NestProg np;
    const double inf = std::numeric_limits<double>::infinity();
    // G[0,20](a0 -> F[0,3] G[0,1] a1): horizon 20 + 3 + 1, memo for F and the inner G
    const std::vector<smc_node> g = {nd(SMC_NODE_ATOM, 0), nd(SMC_NODE_ATOM, 1), nd(SMC_NODE_ALWAYS, 0, 0.0, 1.0),
                                     nd(SMC_NODE_EVENTUALLY, 0, 0.0, 3.0), nd(SMC_NODE_IMPLIES),
                                     nd(SMC_NODE_ALWAYS, 0, 0.0, 20.0)};
    CHECK(compile_n(g, 2, inf, np, err) == SMC_OK);
    CHECK(np.n_nodes == 6 && np.root == 0 && np.height == 5 && !np.unbounded);
    CHECK(np.t_static == 24.0 && np.t_stop == 24.0 && np.n_slots == 2 && slots_ok(np));
    CHECK(np.nd[np.root].kind == SMC_NODE_ALWAYS && np.nd[np.root].slot < 0);

    // the shapes the unit monitor rejects (above) compile here
    // X over F: horizon 1 + 1; F below X has a column
    CHECK(compile_n({nd(SMC_NODE_ATOM, 0), nd(SMC_NODE_EVENTUALLY, 0, 0.0, 1.0), nd(SMC_NODE_NEXT, 0, 0.0, 1.0)}, 1,
                    inf, np, err) == SMC_OK);
    CHECK(np.t_static == 2.0 && np.n_slots == 1 && slots_ok(np));
    // U with a temporal left operand: horizon 2 + max(1, 0)
    CHECK(compile_n({nd(SMC_NODE_ATOM, 0), nd(SMC_NODE_EVENTUALLY, 0, 0.0, 1.0), nd(SMC_NODE_ATOM, 1),
                     nd(SMC_NODE_UNTIL, 0, 0.0, 2.0)},
                    2, inf, np, err) == SMC_OK);
    CHECK(np.t_static == 3.0 && np.n_slots == 1 && slots_ok(np));
    // a nested window with a lower bound: horizon 5 + 2
    CHECK(compile_n({nd(SMC_NODE_ATOM, 0), nd(SMC_NODE_EVENTUALLY, 0, 1.0, 2.0), nd(SMC_NODE_EVENTUALLY, 0, 0.0, 5.0)},
                    1, inf, np, err) == SMC_OK);
    CHECK(np.t_static == 7.0 && np.n_slots == 1 && slots_ok(np));
    // three nested F: horizon 1 + 2 + 3, two columns
    CHECK(compile_n({nd(SMC_NODE_ATOM, 0), nd(SMC_NODE_EVENTUALLY, 0, 0.0, 1.0), nd(SMC_NODE_EVENTUALLY, 0, 0.0, 2.0),
                     nd(SMC_NODE_EVENTUALLY, 0, 0.0, 3.0)},
                    1, inf, np, err) == SMC_OK);
    CHECK(np.t_static == 6.0 && np.n_slots == 2 && np.height == 4 && slots_ok(np));
    // X below F: no column for X (one position per evaluation)
    CHECK(compile_n({nd(SMC_NODE_ATOM, 0), nd(SMC_NODE_NEXT, 0, 0.0, 1.0), nd(SMC_NODE_EVENTUALLY, 0, 0.0, 2.0)}, 1,
                    inf, np, err) == SMC_OK);
    CHECK(np.n_slots == 0 && slots_ok(np));

    // height 10 accepted, 11 rejected (a chain of negations over an F)
    std::vector<smc_node> chain = {nd(SMC_NODE_ATOM, 0), nd(SMC_NODE_EVENTUALLY, 0, 0.0, 1.0)};
    for (int i = 0; i < 8; ++i) chain.push_back(nd(SMC_NODE_NOT));
    CHECK(compile_n(chain, 1, inf, np, err) == SMC_OK && np.height == 10);
    chain.push_back(nd(SMC_NODE_NOT));
    CHECK(compile_n(chain, 1, inf, np, err) == SMC_E_UNSUPPORTED);

    // 32 nodes accepted, 33 rejected: 11 leaves F[0,1+i] a_(i mod 6) joined by
    // 10 ORs in a balanced tree (3 x 11 - 1 = 32 nodes, height 6), then a
    // negation on top
    std::vector<smc_node> wide;
    std::function<void(int, int)> build = [&](int lo, int hi) {
        if (hi - lo == 1) {
            wide.push_back(nd(SMC_NODE_ATOM, lo % 6));
            wide.push_back(nd(SMC_NODE_EVENTUALLY, 0, 0.0, 1.0 + lo));
            return;
        }
        const int mid = (lo + hi) / 2;
        build(lo, mid);
        build(mid, hi);
        wide.push_back(nd(SMC_NODE_OR));
    };
    build(0, 11);
    CHECK(wide.size() == 32 && compile_n(wide, 6, inf, np, err) == SMC_OK && np.n_nodes == 32 && np.height == 6);
    CHECK(np.t_static == 11.0 && np.n_slots == 0 && slots_ok(np));
    wide.push_back(nd(SMC_NODE_NOT));
    CHECK(compile_n(wide, 6, inf, np, err) == SMC_E_UNSUPPORTED);

    // atoms: 6 distinct accepted, 7 rejected
    std::vector<smc_node> six;
    for (int i = 0; i < 6; ++i) {
        six.push_back(nd(SMC_NODE_ATOM, i));
        six.push_back(nd(SMC_NODE_EVENTUALLY, 0, 0.0, 1.0));
        if (i) six.push_back(nd(SMC_NODE_OR));
    }
    CHECK(compile_n(six, 6, inf, np, err) == SMC_OK);
    std::vector<smc_node> seven = six;
    seven.push_back(nd(SMC_NODE_ATOM, 6));
    seven.push_back(nd(SMC_NODE_OR));
    CHECK(compile_n(seven, 7, inf, np, err) == SMC_E_UNSUPPORTED);

    // intervals: 0 <= lo <= hi, lo finite
    const auto f_in_g = [&](double lo, double hi) {
        return std::vector<smc_node>{nd(SMC_NODE_ATOM, 0), nd(SMC_NODE_EVENTUALLY, 0, lo, hi),
                                     nd(SMC_NODE_ALWAYS, 0, 0.0, 1.0)};
    };
    CHECK(compile_n(f_in_g(2.0, 1.0), 1, inf, np, err) == SMC_E_INVALID_ARG);
    CHECK(compile_n(f_in_g(-1.0, 1.0), 1, inf, np, err) == SMC_E_INVALID_ARG);
    CHECK(compile_n(f_in_g(0.0, NAN), 1, inf, np, err) != SMC_OK);
    CHECK(compile_n(f_in_g(inf, inf), 1, inf, np, err) != SMC_OK);
    // unbounded: needs a finite t_max > 0 (the pessimistic rule stops there)
    CHECK(compile_n(f_in_g(0.0, inf), 1, inf, np, err) == SMC_E_INVALID_ARG);
    CHECK(compile_n(f_in_g(0.0, inf), 1, 0.0, np, err) == SMC_E_INVALID_ARG);
    CHECK(compile_n(f_in_g(0.0, inf), 1, 50.0, np, err) == SMC_OK && np.unbounded && np.t_stop == 50.0 &&
          std::isinf(np.t_static));
}

int main()
{
    check_thresholds();
    check_tokens();
    check_formulas();
    check_nested();
    if (failures) {
        printf("failures=%d\n", failures);
        return 1;
    }
    printf("ok\n");
    return 0;
}
