// smc_device.cuh -- device code shared by the generic SSA kernels
// (smc_kernels.cu) and the model-specialized ones compiled at run time
// (smc_jit_kernel.cuh): Philox4x32-10, the uniform maps, the FP64 path's
// logarithm, the compiled BLTLc monitor, instance acquisition, the Wilson
// interval (Eq. 4) and the launch prologue / epilogue.
#pragma once
#include <stdint.h>

#include "smc_internal.h"

#ifndef FULL_MASK
#define FULL_MASK 0xffffffffu
#endif

namespace {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64-bit multiplies with the words permuted and the high halves xored
// with the counter and the round key.  The round keys (key plus multiples of
// the Weyl increments) are uniform over the launch, so they come precomputed
// in the kernel parameters.
__device__ __forceinline__ void philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                         const uint32_t *rk0, const uint32_t *rk1,
                                         uint32_t &w0, uint32_t &w1, uint32_t &w2, uint32_t &w3)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ rk0[r];
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ rk1[r];
        c1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
        c0 = n0;
        c2 = n2;
    }
    w0 = c0; w1 = c1; w2 = c2; w3 = c3;
}

// (0,1) from 52 bits: ((hi:lo) >> 12 + 1/2) 2^-52 = (2v + 1) 2^-53, exact, in
// [2^-53, 1 - 2^-53]: the odd integer 2v + 1 < 2^53 converted exactly, then
// 2^-53 applied to the exponent.  The FP64 event loop never forms it: it
// keeps the odd integer (odd53) and takes -ln u and u a_0 from it.
__device__ __forceinline__ double u01_52(uint32_t hi, uint32_t lo)
{
    const uint64_t n = ((((((uint64_t)hi) << 32) | (uint64_t)lo) >> 12) << 1) | 1ull;
    return __longlong_as_double(__double_as_longlong(__ull2double_rn(n)) - (53ll << 52));
}

// A positive normal float as a double, built on the integer pipe (exact:
// exponent rebiased by 1023 - 127, mantissa shifted into place); anything
// else goes through the conversion instruction.
__device__ __forceinline__ double f32_to_f64(float f)
{
    const uint32_t b = __float_as_uint(f);
    if (__builtin_expect(b - 0x00800000u >= 0x7F000000u, 0)) return (double)f;
    return __hiloint2double((int)((b >> 3) + (896u << 20)), (int)(b << 29));
}

// (0,1) in FP32 from 23 bits: (w >> 9 + 1/2) 2^-23, exact, in [2^-24, 1 - 2^-24].
__device__ __forceinline__ float u01_23(uint32_t w)
{
    return __fmaf_rn((float)(w >> 9), 0x1p-23f, 0x1p-24f);
}

// An integer h as a double (exact for |h| < 2^53, rounded to nearest
// otherwise): on the integer pipes for 0 <= h < 2^53 (fp64i_i2d), else the
// conversion instruction.  GB300's FP64 pipe retires 2 lane-operations per
// clock per SM, so the event loop keeps its conversions off it.
__device__ __forceinline__ double int_to_double(long long h) { return fp64i_i2d(h); }

// The odd integer n = 2v + 1 < 2^53 of the uniform (2v + 1) 2^-53 that
// u01_52(hi, lo) returns (v = the top 52 bits of hi:lo).
__device__ __forceinline__ uint64_t odd53(uint32_t hi, uint32_t lo)
{
    return ((((((uint64_t)hi) << 32) | (uint64_t)lo) >> 12) << 1) | 1ull;
}

// x > y for x, y >= 0 (including +inf): ordered like their bit patterns,
// so the compare runs on the integer pipe.
__device__ __forceinline__ bool dgt(double x, double y)
{
    return __double_as_longlong(x) > __double_as_longlong(y);
}

// ---------------------------------------------------------------------------
// Monitor (one per lane).  Unit semantics, in the knowledge order of the
// event loop (entry times never decrease; after the draw of t' every later
// state has entry time >= t'):
//   witness at a state entered at t:  alive and a <= t <= b and P (and, for
//     nest 1, Q now or later within [t, t + d]; for nest 2, Q at every state
//     entered within [t, t + d]);
//   alive: L held at every earlier state;
//   nest 1 keeps the latest candidate (its window ends last), nest 2 the
//   earliest since the last state violating Q (its window closes first).
// The candidates' entry times live in the lane's shared-memory column tc[u * 32].
struct MonLane {
    long long hb;    // bits of min b over alive undecided units (-1: none)
    uint32_t ab;     // atom bit vector of the current state
    uint32_t alive, pend, done;
    int32_t vidx;    // sum_u value_u 3^u
};

// Register copies of the monitor fields the event loop reads every event;
// the MonLane itself is touched only around the (rare) monitor calls.
struct MonHot {
    long long hb;
    uint32_t pend, ab;
    __device__ __forceinline__ void load(const MonLane &ml)
    {
        hb = ml.hb;
        pend = ml.pend;
        ab = ml.ab;
    }
};

__device__ __constant__ int kPow3[SMC_MAX_UNITS] = {1, 3, 9, 27};

// hb: the draws after which the monitor must be consulted are those whose
// entry time's bit pattern exceeds hb (entry times are >= 0, so hb = -1 means
// every draw): the smallest window end of the alive undecided units, -1 for
// an undecided X unit (its first draw decides or arms it, even at time 0),
// and -1 when no unit is alive.
__device__ __forceinline__ void mon_horizon(MonLane &ml, const MonProg &P)
{
    long long h = 0x7FFFFFFFFFFFFFFFll;
    bool any = false;
#pragma unroll
    for (int u = 0; u < SMC_MAX_UNITS; ++u) {
        if (u < P.n_units && !((ml.done >> u) & 1u) && ((ml.alive >> u) & 1u)) {
            const long long b = P.u[u].nest == 3 ? -1ll : __double_as_longlong(P.u[u].b);
            h = b < h ? b : h;
            any = true;
        }
    }
    ml.hb = any ? h : -1ll;
}

__device__ __forceinline__ void mon_set(MonLane &ml, int u, int val)
{
    ml.done |= 1u << u;
    ml.vidx += val * kPow3[u];
}

// The state just entered at time t (atom bits already in ml.ab).
__device__ __noinline__ int mon_state(MonLane &ml, const MonProg &P, double t, double *tc)
{
    bool changed = false;
#pragma unroll
    for (int u = 0; u < SMC_MAX_UNITS; ++u) {
        if (u >= P.n_units || ((ml.done >> u) & 1u)) continue;
        const MonUnit &U = P.u[u];
        const uint32_t ab = ml.ab;
        const bool l = (U.L >> ab) & 1ull, p = (U.P >> ab) & 1ull, q = (U.Q >> ab) & 1ull;
        bool al = (ml.alive >> u) & 1u, pe = (ml.pend >> u) & 1u;
        if (U.nest == 3) {  // X: pending after a draw within the window, so this is state 1
            if (pe) { mon_set(ml, u, p ? 2 : 1); changed = true; }
            continue;
        }
        const bool inwin = al && !dgt(U.a, t) && !dgt(t, U.b);
        int val = 0;
        if (U.nest == 0) {
            if (inwin && p) val = 2;
        } else if (U.nest == 1) {
            if (pe && q && !dgt(__dsub_rn(t, tc[u * 32]), U.d)) {
                val = 2;
            } else if (inwin && p) {
                if (q) val = 2;
                else { tc[u * 32] = t; pe = true; }
            }
        } else {
            if (pe && !q) pe = false;
            if (inwin && p && q && !pe) { tc[u * 32] = t; pe = true; }
        }
        if (!val) {
            const bool al2 = al && l;
            changed |= (al2 != al);
            al = al2;
            if (!(al && !dgt(t, U.b)) && !pe) val = 1;
        }
        ml.alive = (ml.alive & ~(1u << u)) | ((uint32_t)al << u);
        ml.pend = (ml.pend & ~(1u << u)) | ((uint32_t)pe << u);
        if (val) { mon_set(ml, u, val); changed = true; }
    }
    if (changed) mon_horizon(ml, P);
    return P.table[ml.vidx];
}

// The next state's entry time tn has been drawn (not yet applied).  EXACT =
// false: tn is only a lower bound of that time (a path known up to tmin), so
// an X unit can only be refuted by tn beyond its window.
template <bool EXACT = true>
__device__ __noinline__ int mon_draw(MonLane &ml, const MonProg &P, double tn, const double *tc)
{
    bool changed = false;
#pragma unroll
    for (int u = 0; u < SMC_MAX_UNITS; ++u) {
        if (u >= P.n_units || ((ml.done >> u) & 1u)) continue;
        const MonUnit &U = P.u[u];
        const bool al = (ml.alive >> u) & 1u;
        bool pe = (ml.pend >> u) & 1u;
        if (U.nest == 3) {  // X: the first draw is the next state's entry time
            if (!pe) {
                if ((EXACT && dgt(U.a, tn)) || dgt(tn, U.b)) { mon_set(ml, u, 1); changed = true; }
                else if (EXACT) ml.pend |= 1u << u;
            }
            continue;
        }
        int val = 0;
        if (pe && dgt(__dsub_rn(tn, tc[u * 32]), U.d)) {
            if (U.nest == 2) val = 2;
            else pe = false;
        }
        if (!val && !(al && !dgt(tn, U.b)) && !pe) val = 1;
        ml.pend = (ml.pend & ~(1u << u)) | ((uint32_t)pe << u);
        if (val) { mon_set(ml, u, val); changed = true; }
    }
    if (changed) mon_horizon(ml, P);
    return P.table[ml.vidx];
}

// The path has no further state (absorbing state).
__device__ __noinline__ int mon_close(MonLane &ml, const MonProg &P)
{
#pragma unroll
    for (int u = 0; u < SMC_MAX_UNITS; ++u) {
        if (u >= P.n_units || ((ml.done >> u) & 1u)) continue;
        const bool g_pending = P.u[u].nest == 2 && ((ml.pend >> u) & 1u);
        mon_set(ml, u, g_pending ? 2 : 1);
    }
    return P.table[ml.vidx];
}

__device__ __forceinline__ void mon_start(MonLane &ml, const MonProg &P)
{
    ml.alive = (1u << P.n_units) - 1u;
    ml.pend = 0;
    ml.done = 0;
    ml.vidx = 0;
    mon_horizon(ml, P);
}

// One side of an arithmetic atom: a postfix program over the lane's counts
// (x[i] at xs[i * 32]), FP64, each operation rounded once.
__device__ __forceinline__ double eval_expr(const uint32_t *tk, int n, const int32_t *xs)
{
    double st[SMC_EXPR_MAX_DEPTH + 1];
    int d = 0;
    for (int i = 0; i < n; ++i) {
        const uint32_t w = tk[4 * i];
        const int kind = (int)(w & 255u), arg = (int)(w >> 8);
        double b;
        switch (kind) {
        case SMC_TOK_SPECIES: st[d++] = int_to_double(xs[arg * 32]); break;
        case SMC_TOK_CONST:
            st[d++] = __hiloint2double((int)tk[4 * i + 3], (int)tk[4 * i + 2]);
            break;
        case SMC_TOK_ADD: b = st[--d]; st[d - 1] = __dadd_rn(st[d - 1], b); break;
        case SMC_TOK_SUB: b = st[--d]; st[d - 1] = __dsub_rn(st[d - 1], b); break;
        case SMC_TOK_MUL: b = st[--d]; st[d - 1] = __dmul_rn(st[d - 1], b); break;
        case SMC_TOK_DIV: b = st[--d]; st[d - 1] = __ddiv_rn(st[d - 1], b); break;
        case SMC_TOK_SQRT: st[d - 1] = __dsqrt_rn(st[d - 1]); break;
        default: {
            const double a = st[d - 1];
            double r = 1.0;
            if (arg > 0) {
                r = a;
                for (int k = 1; k < arg; ++k) r = __dmul_rn(r, a);
            }
            st[d - 1] = r;
        }
        }
    }
    return st[0];
}

// An arithmetic atom (record: SMC_ATOM_EXPR, op, token offset, n_lhs, n_rhs).
__device__ __noinline__ uint32_t expr_atom_bit(const uint32_t *A, const uint32_t *ex, const int32_t *xs)
{
    const uint32_t *tk = ex + A[2];
    const int nl = (int)A[3], nr = (int)A[4];
    const double l = eval_expr(tk, nl, xs), r = eval_expr(tk + 4 * nl, nr, xs);
    switch ((int)A[1]) {
    case SMC_OP_LT: return l < r;
    case SMC_OP_LE: return l <= r;
    case SMC_OP_GE: return l >= r;
    case SMC_OP_GT: return l > r;
    case SMC_OP_EQ: return l == r;
    default: return l != r;
    }
}

// Atom a at the lane's current state: L = sum of coef * x over the atom's
// terms (exact int64), bit = (lo <= L <= hi) xor neg, placed at bit a; or
// an arithmetic atom.
template <bool EXT>
__device__ __forceinline__ uint32_t atom_bit(const uint32_t *atoms, const uint32_t *tptr,
                                             const uint32_t *terms, const uint32_t *ex, const int32_t *xs, int a)
{
    const uint32_t *A = atoms + 6 * a;
    const uint32_t w1 = A[0];
    if (EXT && w1 == SMC_ATOM_EXPR) return expr_atom_bit(A, ex, xs) << a;
    long long L;
    if (w1 != 0xFFFFFFFFu) {  // single term
        L = (long long)xs[(w1 & 255u) * 32] * (long long)(((int32_t)w1) >> 8);
    } else {
        L = 0;
        for (uint32_t q = tptr[a], qe = tptr[a + 1]; q < qe; ++q) {
            const uint32_t w = terms[q];
            L += (long long)xs[(w & 255u) * 32] * (long long)(((int32_t)w) >> 8);
        }
    }
    const long long lo = *reinterpret_cast<const long long *>(A + 2);
    const long long hi = *reinterpret_cast<const long long *>(A + 4);
    return (((uint32_t)((L >= lo) & (L <= hi))) ^ A[1]) << a;
}

// ---------------------------------------------------------------------------
// Eq. 4 in FP64, same operation order as the written-out formula:
// (p + z^2/(2n) -+ z sqrt(p(1-p)/n + z^2/(4n^2))) / (1 + z^2/n).
__device__ void wilson_eq4(unsigned long long yes, unsigned long long n, double z, double *out)
{
    if (n == 0) { out[0] = nan(""); out[1] = 0.0; out[2] = 1.0; return; }
    const double dn = (double)n;
    const double p = __ddiv_rn((double)yes, dn);
    const double z2 = __dmul_rn(z, z);
    const double centre = __dadd_rn(p, __ddiv_rn(z2, __dmul_rn(2.0, dn)));
    const double var = __dadd_rn(__ddiv_rn(__dmul_rn(p, __dsub_rn(1.0, p)), dn),
                                 __ddiv_rn(z2, __dmul_rn(__dmul_rn(4.0, dn), dn)));
    const double half = __dmul_rn(z, __dsqrt_rn(var));
    const double den = __dadd_rn(1.0, __ddiv_rn(z2, dn));
    double lo = __ddiv_rn(__dsub_rn(centre, half), den);
    double hi = __ddiv_rn(__dadd_rn(centre, half), den);
    if (yes == 0) lo = 0.0;
    if (yes == n) hi = 1.0;
    out[0] = p;
    out[1] = lo < 0.0 ? 0.0 : lo;
    out[2] = hi > 1.0 ? 1.0 : hi;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}

// Claims an instance for the warp: first one each from the cursor (in the
// launch's list order: the host puts the costliest instances first when it
// knows their costs), then the instance with the most work left --
// trajectories left, times the expected cost of one when known -- so that
// warps whose instance ran dry help the slowest ones.  Returns -1 when no
// work is left.
// Warp-collective.
__device__ int acquire_instance(const SsaParams &p, bool &first, int gw, int lane)
{
    if (first) {
        unsigned i = 0;
        if (lane == 0) i = atomicAdd(p.cursor, 1u);
        i = __shfl_sync(FULL_MASK, i, 0);
        if ((int)i < p.n_list) return p.inst_list[i];
        first = false;
    }
    const int n = p.n_list;
    const int start = (int)(((unsigned)gw * 2654435761u) % (unsigned)n);
    float best = 0.0f;  // trajectories left, times the instance's expected cost when known
    int best_m = -1;
    for (int k = lane; k < n; k += 32) {
        int idx = start + k;
        if (idx >= n) idx -= n;
        const int m = p.inst_list[idx];
        const unsigned long long nx = *((volatile unsigned long long *)&p.tnext[m]);
        const unsigned long long end = p.uniform ? p.u_end : p.tend[m];
        const unsigned long long left = nx < end ? end - nx : 0;
        const float wgt = left ? (float)left * (p.inst_cost ? p.inst_cost[m] : 1.0f) : 0.0f;
        if (wgt > best) { best = wgt; best_m = m; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(FULL_MASK, best, o);
        const int om = __shfl_xor_sync(FULL_MASK, best_m, o);
        if (ob > best || (ob == best && om > best_m)) { best = ob; best_m = om; }
    }
    return best > 0.0f ? best_m : -1;
}

template <bool PLAIN>
struct Prec;
template <>
struct Prec<true> { typedef double T; };
template <>
struct Prec<false> { typedef float T; };

// Block prologue: the monitor program and, on the FP64 path, the
// logarithm's table are copied into the front of shared memory.
__device__ __forceinline__ void stage_block_tables(const SsaParams &p, unsigned char *smem, bool plain)
{
    const uint4 *src = reinterpret_cast<const uint4 *>(p.prog);
    uint4 *dst = reinterpret_cast<uint4 *>(smem);
    for (int i = threadIdx.x; i < (int)(sizeof(MonProg) / 16); i += blockDim.x) dst[i] = src[i];
    if (plain) {
        const uint4 *ls = reinterpret_cast<const uint4 *>(p.logtab);
        uint4 *ld = reinterpret_cast<uint4 *>(smem + sizeof(MonProg));
        for (int i = threadIdx.x; i < p.logtab_bytes / 16; i += blockDim.x) ld[i] = ls[i];
    }
    __syncthreads();
}

// Block epilogue: the last block to finish computes the Wilson interval of
// every instance of the launch.
__device__ __forceinline__ void wilson_epilogue(const SsaParams &p, int *s_last)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned tk = atomicAdd(p.ticket, 1u);
        *s_last = (tk == gridDim.x - 1);
    }
    __syncthreads();
    if (*s_last && p.wilson) {
        __threadfence();
        for (int i = threadIdx.x; i < p.n_list; i += blockDim.x) {
            const int m = p.inst_list[i];
            const volatile unsigned long long *c = p.counts + 4 * m;
            wilson_eq4(c[0], c[1], p.z, p.wilson + 3 * m);
        }
    }
}

}  // namespace
