// smc_kernels.cu -- the persistent SSA + on-the-fly monitor kernel.
//
// One trajectory per thread (the "multiple replications in parallel" policy
// of Sec. 4, one replica per lane instead of one per MPI process).  Each warp
// works on one instance at a time (its model table read through L1); each
// lane keeps its counts x and propensities a in shared-memory columns of the
// warp's slice (lane-minor, so lane i always hits bank i).  Lanes that finish a trajectory claim the next index of the
// instance's work queue by warp ballot (one atomic per refill).
//
// Per event (Sec. 2.2, steps 1-5; Eq. 2a/2b):
//   a0 = sum_j a_j                      (plain: fresh FP64 left-to-right sum;
//                                        mixed: FP32, updated incrementally,
//                                        renormalised in FP64 every 2^k events)
//   (w0..w3) = Philox4x32-10(key = seed, counter = (event, trajectory, instance, 0))
//   tau = -ln(u_tau) / a0,  t' = t + tau (FP64 clock)
//   monitor: windows that t' closes                  (Sec. 3.2: stop as soon as
//   j = first index with running sum > u_sel * a0      the verdict is fixed)
//   x += v_j; a_k recomputed for k in dep(j)
//   monitor: atoms moved by j, then the units at the new state
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "smc.h"
#include "smc_internal.h"

#include "smc_device.cuh"
#include "smc_nest.h"

namespace {


// Rate-law factors of reaction k applied to a (in order): a *= (a0 + a1 x^n)
// / (b0 + b1 x^n), x^n by repeated multiplication, every operation rounded
// once (FP64 path: FP64; mixed path: FP32).
template <bool PLAIN>
__device__ __noinline__ typename Prec<PLAIN>::T apply_factors(typename Prec<PLAIN>::T a, int k,
                                                              const int32_t *xs, const uint32_t *blob)
{
    const uint32_t *fp = blob + blob[BH_FACT_PTR];
    const uint32_t *fw = blob + blob[BH_FACT];
    for (uint32_t q = fp[k], qe = fp[k + 1]; q < qe; ++q) {
        const uint32_t w = fw[q];
        const int32_t x = xs[(w & 255u) * 32];
        const int n = (int)(w >> 8);
        if (PLAIN) {
            const double *c = reinterpret_cast<const double *>(blob + blob[BH_FACT_D]) + 4 * q;
            const double xv = int_to_double(x);
            double xn = xv;
            for (int i = 1; i < n; ++i) xn = __dmul_rn(xn, xv);
            const double num = __dadd_rn(c[0], __dmul_rn(c[1], xn));
            const double den = __dadd_rn(c[2], __dmul_rn(c[3], xn));
            a = (typename Prec<PLAIN>::T)__dmul_rn((double)a, __ddiv_rn(num, den));
        } else {
            const float *c = reinterpret_cast<const float *>(blob + blob[BH_FACT_F]) + 4 * q;
            const float xv = (float)x;
            float xn = xv;
            for (int i = 1; i < n; ++i) xn = __fmul_rn(xn, xv);
            const float num = __fadd_rn(c[0], __fmul_rn(c[1], xn));
            const float den = __fadd_rn(c[2], __fmul_rn(c[3], xn));
            a = (typename Prec<PLAIN>::T)__fmul_rn((float)a, __fdiv_rn(num, den));
        }
    }
    return a;
}

// a_k = c_k h_k(x) (Sec. 2.2) from a propensity word (see smc_internal.h),
// times the reaction's rate-law factors if it has any.  FP64 path: h as an
// exact integer, rounded once; mixed path: h in FP32.
template <bool PLAIN, bool EXT>
__device__ __forceinline__ typename Prec<PLAIN>::T propensity(uint32_t pw, const int32_t *xs,
                                                              const double *rate_d,
                                                              const float *rate_f, const uint32_t *blob)
{
    const int k = pw & 255u, ra = (pw >> 8) & 255u, rb = (pw >> 16) & 255u;
    const int homo = (pw >> 24) & 1u;
    const int32_t xa = xs[ra * 32], xb = xs[rb * 32];
    typename Prec<PLAIN>::T a;
    if (PLAIN) {
        const long long h = ((long long)xa * (long long)(xb - homo)) >> homo;
        a = __dmul_rn(rate_d[k], int_to_double(h));
    } else {
        const float s = homo ? 0.5f : 1.0f;
        const float h = __fmul_rn((float)xa, __fmaf_rn((float)xb, s, homo ? -0.5f : 0.0f));
        a = __fmul_rn(rate_f[k], h);
    }
    if (EXT && (pw & SMC_PW_FACT)) a = apply_factors<PLAIN>(a, k, xs, blob);
    return a;
}

// trace monitor: waiting lanes that make a warp take its pending checks
// together, and the iterations after which it takes them anyway (measured
// on immigration-death with a depth-4 formula, 10^5 trajectories per
// launch: counting due checks too, group 8 / wait 64 0.76M trajectories/s,
// 16 / 256 0.88M, 32 / 128 0.96M, 32 / 512 0.99M, 32 / 2048 1.00M; waiting
// lanes only, 8 / 512 1.18M, 16 / 512 1.18M, 32 / 512 1.20M (1.54M at 10^6
// per launch); a longer wait only delays the early stop of a decided
// trajectory)
#define SMC_NEST_GROUP 32
#define SMC_NEST_WAIT 512

template <bool PLAIN, bool EXT, bool NEST>
__device__ __forceinline__ void run_instance(const SsaParams &p, const MonProg &P, const uint64_t *ltab,
                                             const int m, const uint32_t *blob, int32_t *xs, double *tc,
                                             typename Prec<PLAIN>::T *as, typename Prec<PLAIN>::T *bs,
                                             const int lane)
{
    typedef typename Prec<PLAIN>::T T;
    const int S = (int)blob[BH_S], R = (int)blob[BH_R], NA = (int)blob[BH_NA];
    // selection by checkpoints (SsaParams::sel_block): bs[b * 32] holds the
    // running sum a_0 + ... + a_k at k = 16 b + 15 (or R - 1): the FP64
    // path's exact left-to-right sums, formed with a_0; the mixed path's
    // FP32 block sums a_16b + ... + a_(16b+15), kept along the dependency
    // graph and renormalised with a_0
    const bool blk = p.sel_block != 0 && R > SMC_SEL_BLOCK;
    const int nb = SMC_SEL_BLOCKS(R);
    // mixed path: the block sums from scratch (FP64 sums, rounded once)
    auto block_sums = [&]() {
        for (int b = 0; b < nb; ++b) {
            double s = 0.0;
            for (int k = SMC_SEL_BLOCK * b; k < R && k < SMC_SEL_BLOCK * (b + 1); ++k)
                s = __dadd_rn(s, (double)as[k * 32]);
            bs[b * 32] = (T)s;
        }
    };
    const double *rate_d = reinterpret_cast<const double *>(blob + blob[BH_RATE_D]);
    const float *rate_f = reinterpret_cast<const float *>(blob + blob[BH_RATE_F]);
    const uint32_t *reac = blob + blob[BH_REAC];
    const uint32_t *stp = blob + blob[BH_ST_PTR];
    const uint32_t *st = blob + blob[BH_ST];
    const uint32_t *dpp = blob + blob[BH_DEP_PTR];
    const uint32_t *dp = blob + blob[BH_DEP];
    const uint32_t *amask = blob + blob[BH_AMASK];
    const uint32_t *tptr = blob + blob[BH_ATERM_PTR];
    const uint32_t *terms = blob + blob[BH_ATERM];
    const int32_t *x0 = reinterpret_cast<const int32_t *>(blob + blob[BH_X0]);
    const uint32_t *atoms = blob + blob[BH_ATOM];
    const uint32_t *ex = blob + blob[BH_EXPR];
    const uint32_t *dense = blob + blob[BH_DENSE];
    const bool small = blob[BH_DENSE] != 0;
    const unsigned long long tend = p.uniform ? p.u_end : p.tend[m];
    const bool always_step = P.has_lower != 0;
    const bool unbounded = P.unbounded != 0;
    const double t_max = P.t_max;
    const uint32_t renorm_mask = p.renorm_mask;
    const uint64_t budget = p.budget;

    bool active = false, exhausted = false, snapped = false;
    uint32_t traj = 0, e = 0;
    double t = 0.0;
    T a0 = 0;
    MonLane ml;
    MonHot mh;
    uint32_t c_yes = 0, c_dec = 0, c_bud = 0;
    unsigned long long c_ev = 0;
    const int snap_mode = p.snap_mode;
    const double t_snap = p.t_snap;
    // trace monitor: this lane's recording of the trajectory, and the
    // doubling schedule of its checks (events 0, 1, 2, 4, ...; also at the
    // horizon, absorption and the budget)
    const NestProg *NP = NEST ? p.nest : nullptr;  // (NEST: a kernel variant of its own)
    const uint64_t lane_id = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t cap = p.tr_cap;  // this lane's positions are contiguous
    double *trt = NP ? p.tr_t + lane_id * cap : nullptr;
    uint32_t *trw = NP ? p.tr_w + lane_id * cap : nullptr;
    const int n_slots = (NP && p.tr_m) ? NP->n_slots : 0;
    uint32_t *trm = n_slots ? p.tr_m + lane_id * n_slots * cap : nullptr;
    // a recorded position's memo cells start unknown
    auto clear_memo = [&](uint32_t pos) {
        for (int k = 0; k < n_slots; ++k) trm[k * cap + pos] = 0u;
    };
    uint64_t nchk = 0;
    // Checks are taken by the warp's lanes together (the evaluation's loops
    // then run side by side instead of one lane at a time): a lane whose
    // check would end its trajectory one way or another waits (hold: 1 the
    // horizon draw, entry time hold_t; 2 absorbed; 3 at the event budget),
    // one on the doubling schedule keeps simulating (due); the waiting and
    // due lanes evaluate when SMC_NEST_GROUP lanes wait, when every active
    // lane waits, or SMC_NEST_WAIT iterations after a check became pending
    // (due checks ride along: they stop a decided trajectory early, but
    // need not be taken at once).  `passed`: the event whose horizon check
    // came back undecided on a bounded formula (its draw is then taken).
    int hold = 0;
    double hold_t = 0.0;
    bool due = false;
    uint32_t passed = 0xFFFFFFFFu;
    int wait_it = 0;

    // verdict codes: 1 false, 2 true, 3 event budget exhausted, 4 stopped at
    // the snapshot (prefix-only run: no verdict, not counted), 5 trace
    // monitor gave up (its recording full, or still undecided when the
    // clock passed 4 t_stop + 1): counted with the budget's undecided ones
    auto finish = [&](int v) {
        if (v == 3 || v == 5) ++c_bud;
        else if (v != 4) { ++c_dec; c_yes += (v == 2); }
        c_ev += e;
        const uint64_t idx = (uint64_t)m * p.out_stride + ((uint64_t)traj - p.out_base);
        if (p.o_verdict) {
            p.o_verdict[idx] = (v == 2);
            if (p.o_status) p.o_status[idx] = (v == 3) ? 1 : (v == 4 ? 2 : (v == 5 ? 3 : 0));
            if (p.o_events) p.o_events[idx] = e;
            if (p.o_tfinal) p.o_tfinal[idx] = t;
            if (p.o_xfinal)
                for (int i = 0; i < S; ++i) p.o_xfinal[idx * p.x_stride + i] = xs[i * 32];
        }
        if (snap_mode && !snapped) {  // decided before t_snap
            p.o_snap[idx] = 1;
            if (p.o_esnap) p.o_esnap[idx] = e;
        }
        active = false;
    };
    // trace monitor: the formula on the recorded positions 0..e and what
    // follows them (smc_nest.h)
    auto nest_at = [&](int end, double tnx) -> NestVal {
        const NestTrace T{trt, trw, 1, (int64_t)e, end, tnx, trm, (int64_t)cap};
        return nest_decide(*NP, T);
    };
    // stop at the decision point: the trajectory's outputs are those of
    // position k = d / 2 (the counts rewound by the reactions recorded after it)
    auto finish_at = [&](NestVal d) {
        const uint32_t k = (uint32_t)(d.d >> 1);
        if (p.o_xfinal)
            for (uint32_t m2 = e; m2 > k; --m2) {
                const uint32_t jr = trw[m2] >> 24;
                for (uint32_t q = stp[jr], qe = stp[jr + 1]; q < qe; ++q) {
                    const uint32_t w = st[q];
                    xs[(w & 255u) * 32] -= ((int32_t)w) >> 8;
                }
            }
        e = k;
        t = trt[k];
        finish(d.v);
    };

    for (;;) {
        // one vote per iteration: which lanes hold a trajectory
        unsigned act = __ballot_sync(FULL_MASK, active);
        if (!exhausted && act != FULL_MASK) {
            const unsigned need = ~act;
            const int nneed = __popc(need);
            if (nneed >= p.refill || nneed == 32) {
                const int leader = __ffs(need) - 1;
                unsigned long long base = 0;
                if (lane == leader) base = atomicAdd(&p.tnext[m], (unsigned long long)nneed);
                base = __shfl_sync(FULL_MASK, base, leader);
                if (base + (unsigned long long)nneed >= tend) exhausted = true;
                if (!active) {
                    const unsigned long long id = base + __popc(need & ((1u << lane) - 1u));
                    if (id < tend) {
                        // start trajectory `id`: x = x0 (plus the constant-1
                        // column), fresh propensities, monitor at t = 0
                        traj = (uint32_t)id;
                        e = 0;
                        t = 0.0;
                        snapped = false;
                        for (int i = 0; i < S; ++i) xs[i * 32] = x0[i];
                        xs[S * 32] = 1;
                        double s = 0.0;
                        for (int k = 0; k < R; ++k) {
                            const T ak = propensity<PLAIN, EXT>(reac[k], xs, rate_d, rate_f, blob);
                            as[k * 32] = ak;
                            s = __dadd_rn(s, (double)ak);
                        }
                        a0 = (T)s;
                        if (!PLAIN && blk) block_sums();
                        uint32_t ab = 0;
                        for (int a = 0; a < NA; ++a) ab |= atom_bit<EXT>(atoms, tptr, terms, ex, xs, a);
                        active = true;
                        if constexpr (NEST) {
                            trt[0] = 0.0;
                            trw[0] = ab;
                            clear_memo(0);
                            mh.ab = ab;
                            nchk = 1;
                            hold = 0;
                            due = false;
                            passed = 0xFFFFFFFFu;
                            const NestVal d = nest_at(0, 0.0);
                            if (d.v) finish_at(d);
                        } else {
                            ml.ab = ab;
                            mon_start(ml, P);
                            const int v = mon_state(ml, P, 0.0, tc);
                            mh.load(ml);
                            if (v) finish(v);
                        }
                    }
                }
                act = __ballot_sync(FULL_MASK, active);
            }
        }
        if (!act) {
            if (exhausted) break;
            continue;
        }
        if constexpr (NEST) {  // the pending checks, taken together
            const unsigned H = __ballot_sync(FULL_MASK, active && hold != 0);
            const unsigned W = __ballot_sync(FULL_MASK, active && (hold != 0 || due));
            if (W) ++wait_it;
            if (H == act || __popc(H) >= SMC_NEST_GROUP || wait_it >= SMC_NEST_WAIT) {
                wait_it = 0;
                if (active && (hold != 0 || due)) {
                    const int h = hold;
                    hold = 0;
                    due = false;
                    const NestVal d = nest_at(h == 1 ? 1 : (h == 2 ? 2 : 0), hold_t);
                    if (d.v) {
                        finish_at(d);
                    } else if (h == 1) {
                        if (NP->unbounded) finish_at(NestVal{1, 2 * (int64_t)e + 1});  // pessimistic rule
                        else if (dgt(hold_t, __dadd_rn(__dmul_rn(4.0, NP->t_stop), 1.0))) finish(5);
                        else passed = e;  // resume: take the draw
                    } else if (h == 2) {
                        finish(5);
                    } else if (h == 3) {
                        finish(3);
                    }
                }
                continue;
            }
            if (hold != 0) continue;
        }
        if (!active) continue;

        // ---- one event -------------------------------------------------------
        T pre[SMC_SMALL_MAX];  // small networks: running sums a_0 + ... + a_k
        uint32_t pos = 0;      // small networks: bit k set iff a_k > 0
        if (small) {  // step 1 from scratch: every propensity of the current state
            T acc = (T)0;
#pragma unroll
            for (int k = 0; k < SMC_SMALL_MAX; ++k) {
                if (k < R) {
                    const T ak = propensity<PLAIN, EXT>(reac[k], xs, rate_d, rate_f, blob);
                    const bool positive =
                        PLAIN ? __double_as_longlong((double)ak) > 0 : ak > (T)0;
                    pos |= (uint32_t)positive << k;
                    acc = PLAIN ? (T)__dadd_rn((double)acc, (double)ak) : (T)__fadd_rn((float)acc, (float)ak);
                    pre[k] = acc;
                }
            }
            a0 = acc;
        } else if (PLAIN) {  // step 1: a0 as a fresh left-to-right sum
            double s = 0.0;
            if (blk) {  // keeping the running sum at the end of every block
                for (int b = 0; b < nb; ++b) {
                    for (int k = SMC_SEL_BLOCK * b; k < R && k < SMC_SEL_BLOCK * (b + 1); ++k)
                        s = __dadd_rn(s, (double)as[k * 32]);
                    bs[b * 32] = (T)s;
                }
            } else {
                for (int k = 0; k < R; ++k) s = __dadd_rn(s, (double)as[k * 32]);
            }
            a0 = (T)s;
        } else if (!(a0 > (T)0)) {  // drifted running sum: renormalise in FP64
            double s = 0.0;
            for (int k = 0; k < R; ++k) s = __dadd_rn(s, (double)as[k * 32]);
            a0 = (T)s;
            if (blk) block_sums();
        }
        if (PLAIN ? __double_as_longlong((double)a0) <= 0 : !(a0 > (T)0)) {  // absorbing state: no further position
            if constexpr (NEST) {
                hold = 2;
            } else {
                finish(mon_close(ml, P));
            }
            continue;
        }
        uint32_t w0, w1, w2, w3;
        philox10(e, traj, (uint32_t)m, 0u, p.rk0, p.rk1, w0, w1, w2, w3);
        double tn;
        T r;
        if (PLAIN) {
            // tau = -ln u01_52(w0, w1) / a_0 rounded once on the integer pipes
            uint64_t sm;
            int lz;
            fp64i_neglog53_norm(odd53(w0, w1), ltab, sm, lz);
            tn = __dadd_rn(t, fp64i_tau(sm, lz, (double)a0));
            r = (T)__dmul_rn(u01_52(w2, w3), (double)a0);
        } else {
            const float ut = u01_23(w0), us = u01_23(w2);
            const float tau = __fdividef(-__logf(ut), (float)a0);
            tn = __dadd_rn(t, f32_to_f64(tau));
            r = (T)__fmul_rn(us, (float)a0);
        }
        if (snap_mode && !snapped && dgt(tn, t_snap)) {
            // the current state is the one occupied at t_snap, and the
            // verdict was not fixed by anything known up to t_snap
            snapped = true;
            const uint64_t idx = (uint64_t)m * p.out_stride + ((uint64_t)traj - p.out_base);
            p.o_snap[idx] = 0;
            if (p.o_esnap) p.o_esnap[idx] = e;
            for (int i = 0; i < S; ++i) p.o_xsnap[idx * p.x_stride + i] = xs[i * 32];
            if (snap_mode == 2) { finish(4); continue; }
        }
        int v = 0;
        if constexpr (NEST) {
            if (dgt(tn, NP->t_stop) && passed != e) {  // no later position can matter (or, unbounded: t_max passed)
                hold = 1;
                hold_t = tn;
                continue;
            }
        } else {
            if (mh.pend || __double_as_longlong(tn) > mh.hb) {
                v = mon_draw(ml, P, tn, tc);
                mh.load(ml);
            }
            if (!v && unbounded && dgt(tn, t_max)) v = 1;  // pessimistic rule (Sec. 3.2)
            if (v) { finish(v); continue; }
        }

        // step 2: selection, first j whose running sum exceeds r
        int j = -1, last = -1;
        if (small) {  // the running sums are already in registers
#pragma unroll
            for (int k = 0; k < SMC_SMALL_MAX; ++k) {
                const bool hit = PLAIN ? __double_as_longlong((double)pre[k]) >
                                             __double_as_longlong((double)r)
                                       : pre[k] > r;
                if (k < R && j < 0 && hit) j = k;
            }
            last = pos ? 31 - __clz(pos) : -1;
        } else if (PLAIN && blk) {
            // the first block whose closing running sum exceeds r holds j;
            // the sum restarts from the previous checkpoint, so every running
            // sum is the left-to-right one of the linear scan, bit for bit
            const long long rb = __double_as_longlong((double)r);
            int b = 0;
            while (b < nb && __double_as_longlong((double)bs[b * 32]) <= rb) ++b;
            if (b < nb) {
                double cum = b ? (double)bs[(b - 1) * 32] : 0.0;
                for (int k = SMC_SEL_BLOCK * b; k < R && k < SMC_SEL_BLOCK * (b + 1); ++k) {
                    cum = __dadd_rn(cum, (double)as[k * 32]);
                    if (__double_as_longlong(cum) > rb) { j = k; break; }
                }
            } else {
                for (int k = R - 1; k >= 0 && last < 0; --k)
                    if (__double_as_longlong((double)as[k * 32]) > 0) last = k;
            }
        } else if (PLAIN) {
            const long long rb = __double_as_longlong((double)r);
            double cum = 0.0;
            for (int k = 0; k < R; ++k) {
                const double ak = (double)as[k * 32];
                cum = __dadd_rn(cum, ak);
                if (__double_as_longlong(ak) > 0) last = k;
                if (__double_as_longlong(cum) > rb) { j = k; break; }
            }
        } else if (blk) {
            float cum = 0.0f;
            int b = 0;
            for (; b < nb; ++b) {
                const float nc = cum + (float)bs[b * 32];
                if (nc > (float)r) break;
                cum = nc;
            }
            if (b < nb) {
                for (int k = SMC_SEL_BLOCK * b; k < R && k < SMC_SEL_BLOCK * (b + 1); ++k) {
                    const float ak = (float)as[k * 32];
                    cum += ak;
                    if (ak > 0.0f) last = k;
                    if (cum > (float)r) { j = k; break; }
                }
            }
            if (j < 0)
                for (int k = R - 1; k >= 0 && last < 0; --k)
                    if ((float)as[k * 32] > 0.0f) last = k;
        } else {
            float cum = 0.0f;
            for (int k = 0; k < R; ++k) {
                const float ak = (float)as[k * 32];
                cum += ak;
                if (ak > 0.0f) last = k;
                if (cum > (float)r) { j = k; break; }
            }
        }
        if (j < 0) j = last;  // r reached the full sum (rounding, or a drifted a0)
        if (j < 0) {          // every a_k is 0 (only a drifted FP32 a0 gets here)
            if constexpr (NEST) {
                hold = 2;
            } else {
                finish(mon_close(ml, P));
            }
            continue;
        }

        // step 4: x += v_j, then the propensities that read a changed species
        uint32_t ab = mh.ab;
        if (small) {  // dense byte row of v_j; atoms re-evaluated in full
            const uint32_t d0 = dense[2 * j], d1 = dense[2 * j + 1];
#pragma unroll
            for (int i = 0; i < SMC_SMALL_MAX; ++i)
                if (i < S) xs[i * 32] += (int32_t)(int8_t)((i < 4 ? d0 : d1) >> (8 * (i & 3)));
            ++e;
            t = tn;
            ab = 0;
            for (int a = 0; a < NA; ++a) ab |= atom_bit<EXT>(atoms, tptr, terms, ex, xs, a);
        } else {
            for (uint32_t q = stp[j], qe = stp[j + 1]; q < qe; ++q) {
                const uint32_t w = st[q];
                xs[(w & 255u) * 32] += ((int32_t)w) >> 8;
            }
            for (uint32_t q = dpp[j], qe = dpp[j + 1]; q < qe; ++q) {
                const uint32_t pw = dp[q];
                const int k = pw & 255u;
                const T ak = propensity<PLAIN, EXT>(pw, xs, rate_d, rate_f, blob);
                if (!PLAIN) {
                    const T d = ak - as[k * 32];
                    a0 = a0 + d;
                    if (blk) bs[(k / SMC_SEL_BLOCK) * 32] += d;
                }
                as[k * 32] = ak;
            }
            ++e;
            t = tn;
            if (!PLAIN && (e & renorm_mask) == 0u) {  // FP64 renormalisation of a0
                double s = 0.0;
                for (int k = 0; k < R; ++k) s = __dadd_rn(s, (double)as[k * 32]);
                a0 = (T)s;
                if (blk) block_sums();
            }
            // monitor at the new state: re-evaluate the atoms that j moves
            uint32_t am = amask[j];
            while (am) {
                const int a = __ffs(am) - 1;
                am &= am - 1u;
                ab = (ab & ~(1u << a)) | atom_bit<EXT>(atoms, tptr, terms, ex, xs, a);
            }
        }
        if constexpr (NEST) {  // record the new position; check on the doubling schedule and at the budget
            if (e >= p.tr_cap) { finish(5); continue; }
            trt[e] = t;
            trw[e] = ab | ((uint32_t)j << 24);
            clear_memo(e);
            mh.ab = ab;
            if ((uint64_t)e >= budget) hold = 3;
            else if ((uint64_t)e == nchk) {
                due = true;
                nchk *= 2;
            }
            continue;
        }
        if (always_step || ab != mh.ab || mh.pend) {
            ml.ab = ab;
            v = mon_state(ml, P, t, tc);
            mh.load(ml);
        }
        if (v) finish(v);
        else if ((uint64_t)e >= budget) finish(3);
    }

    // warp reduction of the instance's counts, one atomic per counter
    const unsigned long long s_yes = warp_sum(c_yes), s_dec = warp_sum(c_dec);
    const unsigned long long s_ev = warp_sum(c_ev), s_bud = warp_sum(c_bud);
    if (lane == 0 && (s_dec | s_bud)) {
        atomicAdd(&p.counts[4 * m + 0], s_yes);
        atomicAdd(&p.counts[4 * m + 1], s_dec);
        atomicAdd(&p.counts[4 * m + 2], s_ev);
        atomicAdd(&p.counts[4 * m + 3], s_bud);
    }
}

// Register budget: 64 per thread for the mixed path (32 resident warps per
// SM), 80 for the FP64 path (24 warps; its FP64 pipe saturates before issue).
// EXT: the model uses rate-law factors or arithmetic atoms; without them the
// kernel carries none of their code (and none of its register pressure).
template <bool PLAIN, bool EXT, bool NEST>
__global__ void __launch_bounds__(256, PLAIN ? 3 : 4) ssa_kernel(const SsaParams p)
{
    typedef typename Prec<PLAIN>::T T;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_last;
    stage_block_tables(p, smem, PLAIN);  // monitor program, then the logarithm's table
    const MonProg &P = *reinterpret_cast<const MonProg *>(smem);
    const uint64_t *ltab = reinterpret_cast<const uint64_t *>(smem + sizeof(MonProg));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // warp slice: x[(s_max + 1)][32] | tc[units][32] | a[r_max][32]; the
    // instance's table is read from global memory through L1, where it stays
    // while the warp works on that instance (shared memory holding it cost
    // occupancy: measured 7.7M vs 8.9M trajectories/s on 4096 networks)
    unsigned char *wb = smem + sizeof(MonProg) + p.logtab_bytes + (size_t)warp * p.warp_bytes;
    const uint32_t *blob = nullptr;
    unsigned char *lanes = wb;
    int32_t *xs = reinterpret_cast<int32_t *>(lanes) + lane;
    lanes += (size_t)(p.s_max + 1) * 128;
    double *tc = reinterpret_cast<double *>(lanes) + lane;
    lanes += (size_t)p.tc_bytes;
    T *as = reinterpret_cast<T *>(lanes) + lane;
    T *bs = as + (size_t)p.r_max * 32;  // checkpoints (blocked selection only)

    bool first = true;
    int cur = -1;
    const int gw = blockIdx.x * (blockDim.x >> 5) + warp;
    for (;;) {
        const int m = acquire_instance(p, first, gw, lane);
        if (m < 0) break;
        if (m != cur) {
            blob = p.blobs + p.blob_off[m];
            cur = m;
        }
        run_instance<PLAIN, EXT, NEST>(p, P, ltab, m, blob, xs, tc, as, bs, lane);
        __syncwarp();
    }

    wilson_epilogue(p, &s_last);
}

__global__ void queue_init_kernel(const SsaParams p)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < p.n_inst) p.tnext[i] = p.uniform ? p.u_begin : p.tbegin[i];
    if (i == 0) { *p.cursor = 0u; *p.ticket = 0u; }
}

// Replays given paths through the compiled monitor (one thread per path).
// decided_at is the point where the verdict was fixed: 2k after state k was
// processed, 2k+1 after the entry time of state k+1 (or, after the last
// state, tmin / the end of the path) was known.
__global__ void replay_kernel(const ReplayParams rp)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rp.n_paths) return;
    const MonProg &P = *rp.prog;
    const int na = P.n_atoms, S = rp.S, n = rp.len[i];
    const int32_t *x = rp.x + rp.off[i] * S;
    const double *t = rp.t + rp.off[i];
    if (rp.nest) {  // trace monitor: the path as recorded, then what follows it
        uint32_t *w = rp.w + rp.off[i];
        for (int k = 0; k < n; ++k) {
            uint32_t ab = 0;
            for (int a = 0; a < na; ++a) {
                long long L = 0;
                for (int s2 = 0; s2 < S; ++s2) L += (long long)rp.coef[a * S + s2] * x[k * S + s2];
                const uint32_t in = (L >= rp.athr[2 * a]) & (L <= rp.athr[2 * a + 1]);
                ab |= (in ^ ((rp.aneg >> a) & 1u)) << a;
            }
            w[k] = ab;
        }
        const NestTrace T{t, w, 1, (int64_t)n - 1, rp.closed[i] ? 2 : 3, rp.tmin[i]};
        const NestVal d = nest_decide(*rp.nest, T);
        rp.verdict[i] = d.v;
        rp.decided_at[i] = d.v ? d.d : -1;
        return;
    }
    double tc_local[SMC_MAX_UNITS * 32];
    double *tc = tc_local;
    MonLane ml;
    int v = 0;
    long long q = -1;
    for (int k = 0; k < n && !v; ++k) {
        if (k > 0) {
            if (ml.pend || __double_as_longlong(t[k]) > ml.hb) v = mon_draw(ml, P, t[k], tc);
            if (v) { q = 2 * k - 1; break; }
        }
        uint32_t ab = 0;
        for (int a = 0; a < na; ++a) {
            long long L = 0;
            for (int s = 0; s < S; ++s) L += (long long)rp.coef[a * S + s] * x[k * S + s];
            const uint32_t in = (L >= rp.athr[2 * a]) & (L <= rp.athr[2 * a + 1]);
            ab |= (in ^ ((rp.aneg >> a) & 1u)) << a;
        }
        ml.ab = ab;
        if (k == 0) mon_start(ml, P);
        v = mon_state(ml, P, t[k], tc);
        if (v) q = 2 * k;
    }
    if (!v && n > 0) {
        if (rp.closed[i]) v = mon_close(ml, P);
        else v = mon_draw<false>(ml, P, rp.tmin[i], tc);  // tmin bounds the next entry time
        if (v) q = 2 * (long long)n - 1;
    }
    rp.verdict[i] = v;
    rp.decided_at[i] = q;
}

}  // namespace

// ---------------------------------------------------------------------------
// host wrappers

// The last error of a launch wrapper below (its text for the host's messages:
// cudaGetLastError, once read, no longer holds it).
static thread_local cudaError_t g_kernel_err = cudaSuccess;

static int to_code(cudaError_t e)
{
    if (e != cudaSuccess) g_kernel_err = e;
    return e == cudaSuccess ? 0 : -3;
}

const char *smc_kernel_error() { return cudaGetErrorString(g_kernel_err); }

// variant: bit 0 rate-law factors or arithmetic atoms (EXT), bit 1 the
// trace monitor (NEST)
static const void *ssa_kernel_ptr(int plain, int variant)
{
    const void *k[2][4] = {{(const void *)ssa_kernel<false, false, false>, (const void *)ssa_kernel<false, true, false>,
                            (const void *)ssa_kernel<false, false, true>, (const void *)ssa_kernel<false, true, true>},
                           {(const void *)ssa_kernel<true, false, false>, (const void *)ssa_kernel<true, true, false>,
                            (const void *)ssa_kernel<true, false, true>, (const void *)ssa_kernel<true, true, true>}};
    return k[plain ? 1 : 0][variant & 3];
}

int smc_ssa_set_smem_limit(int plain, int ext, int smem_bytes)
{
    return to_code(cudaFuncSetAttribute(ssa_kernel_ptr(plain, ext), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        smem_bytes));
}

int smc_ssa_max_blocks_per_sm(int plain, int ext, int block, int smem_bytes, int *out)
{
    return to_code(cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, ssa_kernel_ptr(plain, ext), block, smem_bytes));
}

int smc_launch_ssa(int plain, int ext, const SsaParams &p, int grid, int block, int smem_bytes, void *stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    void *args[] = {(void *)&p};
    return to_code(cudaLaunchKernel(ssa_kernel_ptr(plain, ext), dim3(grid), dim3(block), args, (size_t)smem_bytes, s));
}

int smc_launch_queue_init(const SsaParams &p, void *stream)
{
    const int n = p.n_inst > 0 ? p.n_inst : 1;
    queue_init_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(p);
    return to_code(cudaGetLastError());
}

int smc_launch_replay(const ReplayParams &rp, void *stream)
{
    const int n = rp.n_paths > 0 ? rp.n_paths : 1;
    replay_kernel<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(rp);
    return to_code(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// The FP64 path's logarithm and division on arrays (tests and callers that
// want the same functions).
__global__ void log_batch_kernel(const uint64_t *tab_g, const double *u, uint64_t n, double *out)
{
    __shared__ uint64_t tab[SMC_LOGTAB_BYTES / 8];
    for (int i = threadIdx.x; i < SMC_LOGTAB_BYTES / 8; i += blockDim.x) tab[i] = tab_g[i];
    __syncthreads();
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = fp64i_log(u[i], tab);
}

int smc_launch_log_batch(const uint64_t *tab, const double *u, uint64_t n, double *out, void *stream)
{
    if (n == 0) return 0;
    const unsigned blocks = (unsigned)std::min<uint64_t>(4096, (n + 255) / 256);
    log_batch_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(tab, u, n, out);
    return to_code(cudaGetLastError());
}

__global__ void div_batch_kernel(const double *num, const double *den, uint64_t n, double *out)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = fp64i_div(num[i], den[i]);
}

int smc_launch_div_batch(const double *num, const double *den, uint64_t n, double *out, void *stream)
{
    if (n == 0) return 0;
    const unsigned blocks = (unsigned)std::min<uint64_t>(4096, (n + 255) / 256);
    div_batch_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(num, den, n, out);
    return to_code(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Snapshot features: row (m, k) = x_snap / x_scale, t_snap / t_scale, the
// instance's centred log rate constants (zero for rows without a snapshot).
// Row (m, k): the chosen species' counts scaled (Fs values, species sidx[i]),
// the time, then R log-rate features of instance m (R = 0: none).
__global__ void snapshot_features_kernel(uint64_t n_rows, uint64_t n_traj, int Fs, const int32_t *sidx, int R,
                                         int x_stride, const int32_t *x_snap, const float *x_scale, float t_feat,
                                         const float *lograte, float *feat)
{
    const uint64_t row = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n_rows) return;
    const uint64_t m = row / n_traj;
    const int F = Fs + 1 + R;
    float *f = feat + row * F;
    for (int i = 0; i < Fs; ++i) f[i] = (float)x_snap[row * x_stride + sidx[i]] / x_scale[i];
    f[Fs] = t_feat;
    for (int j = 0; j < R; ++j) f[Fs + 1 + j] = lograte[m * R + j];
}

int smc_launch_snapshot_features(uint64_t n_rows, uint64_t n_traj, int Fs, const int32_t *sidx, int R,
                                 int x_stride, const int32_t *x_snap, const float *x_scale, float t_feat,
                                 const float *lograte, float *feat, void *stream)
{
    if (n_rows == 0) return 0;
    snapshot_features_kernel<<<(unsigned)((n_rows + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        n_rows, n_traj, Fs, sidx, R, x_stride, x_snap, x_scale, t_feat, lograte, feat);
    return to_code(cudaGetLastError());
}

// Control-variate sums over n trajectories: G = g for trajectories alive at
// the snapshot, G = Y for those decided before it; sums[0..6] += (count,
// sum Y, sum G, sum Y^2, sum G^2, sum Y G, sum e_pre) in FP64 (Y ignored for
// prefix-only runs, whose verdict is unknown: they contribute count and the G
// sums, with G = Y only when decided before the snapshot; e_pre, the events
// up to the snapshot or the verdict, may be null).
__global__ void cv_sums_kernel(uint64_t n, const uint8_t *y, const uint8_t *snap, const float *g,
                               const uint32_t *e_pre, int prefix, double *sums)
{
    double s[7] = {0, 0, 0, 0, 0, 0, 0};
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const double Y = y[i];
        const double G = snap[i] ? Y : (double)g[i];
        s[0] += 1.0;
        s[1] += prefix ? 0.0 : Y;
        s[2] += G;
        s[3] += prefix ? 0.0 : Y * Y;
        s[4] += G * G;
        s[5] += prefix ? 0.0 : Y * G;
        s[6] += e_pre ? (double)e_pre[i] : 0.0;  // what a prefix-only run of this trajectory costs
    }
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        double v = s[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&sums[k], v);
    }
}

int smc_launch_cv_sums(uint64_t n, const uint8_t *y, const uint8_t *snap, const float *g, const uint32_t *e_pre,
                       int prefix, double *sums, void *stream)
{
    if (n == 0) return 0;
    const unsigned blocks = (unsigned)std::min<uint64_t>(1024, (n + 255) / 256);
    cv_sums_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(n, y, snap, g, e_pre, prefix, sums);
    return to_code(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Scratch of smc_simulate_noalloc: the SSA kernel's work queue (one 64-bit
// counter per instance) followed by its instance cursor and finish ticket,
// in a fixed array that every GPU loading this library holds until the
// process exits (SMC_NOALLOC_MAX_INSTANCES + 2 words, about 32 KiB).  It is
// shared by every call on a device: each call resets the counters it uses
// (queue_init_kernel) before its SSA launch, and calls whose launches
// overlap on the GPU race on it.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[SMC_NOALLOC_MAX_INSTANCES + 2];

// Device address of the array on `device`, which must be the current
// device.  Looked up with cudaGetSymbolAddress on the first call per device
// (host code may not use the array's name as an address) and cached.
int smc_noalloc_scratch(int device, unsigned long long **queue, unsigned int **sync)
{
    static std::mutex mu;
    static unsigned long long *addr[SMC_NOALLOC_MAX_DEVICES] = {};
    if (device < 0 || device >= SMC_NOALLOC_MAX_DEVICES || !queue || !sync) return -1;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return -3;
        addr[device] = static_cast<unsigned long long *>(p);
    }
    *queue = addr[device];
    *sync = reinterpret_cast<unsigned int *>(addr[device] + SMC_NOALLOC_MAX_INSTANCES);
    return 0;
}
