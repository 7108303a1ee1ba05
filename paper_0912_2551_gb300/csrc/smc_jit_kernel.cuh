// smc_jit_kernel.cuh -- the persistent SSA + monitor kernel specialized to one
// network structure, compiled at run time (NVRTC) when a model is loaded.
//
// The generated header "smc_jit_model.h" fixes the structure as code:
//   JS, JR, JNA                  species, reactions, atoms
//   jit_props_plain / _mixed     a_k = c_k h_k(x) for every k, their running
//                                sums (the selection table of Eq. 2b) and the
//                                bit set of positive a_k
//   jit_apply(j, x, sgn)         x += sgn v_j
//   jit_atoms(x)                 the atom bit vector of the monitor
// so each lane keeps its counts x in registers and no table is read per
// event.  Rates (and x0) stay data, read once per instance, so one compiled
// kernel serves every parameter set of the structure.  The arithmetic, its
// order and the random-number use are those of the generic kernel's
// small-network branch: both produce the same trajectories bit for bit.
#pragma once
#include "smc_device.cuh"
#include "smc_jit_model.h"

// Medium networks (JIT_MEDIUM: more than 8 species or reactions): the fired
// reaction's net changes come from kJitDelta staged in shared memory (one
// row of JW words per reaction), the rates from a per-warp shared-memory
// slice, and the launch keeps 2 blocks of 256 threads per SM (128 registers
// per thread for the counts and the prefix sums).
#ifdef JIT_MEDIUM
#define JIT_DELTA_BYTES ((JR * JW * 4 + 15) / 16 * 16)
#define JIT_MINB_PLAIN 2
#define JIT_MINB_MIXED 2
#else
#define JIT_DELTA_BYTES 0
#define JIT_MINB_PLAIN 3
#define JIT_MINB_MIXED 4
#endif

// The tail of a launch: when a warp's queue is drained and one trajectory is
// left, its 32 lanes advance that trajectory several events per round by
// speculating over the reactions fired (small networks): lane 0 takes the
// event from the current state; lanes 1..JR the next one after reaction
// k = lane - 1; with JR <= 5, lanes 1+JR..JR+JR^2 the one after that for
// the reaction pair ((lane-1-JR) / JR, (lane-1-JR) % JR).  The realized path
// then picks its lanes' results in order; the arithmetic of every event is
// the sequential one, so trajectories are unchanged.
#ifndef JIT_MEDIUM
#define JIT_COOP_DEPTH (JR <= 5 ? 2 : 1)
#endif

namespace {

// One event's random numbers (Sec. 2.2, step 2 and Eq. 2a): -ln u_tau and
// u_sel from the Philox block of (event e, trajectory, instance).  They
// depend on the event index alone, so the kernel draws them one event ahead
// and the logarithm leaves the chain that runs through the counts.
// FP64 path: -ln u_tau as the normalised 64-bit value of fp64i_neglog53_norm
// (sm, lz), so that tau is formed on the integer pipes (fp64i_tau), and
// u_sel as a double.
template <bool PLAIN>
struct JitDraw;
template <>
struct JitDraw<true> {
    uint64_t sm;
    double us;
    int lz;
};
template <>
struct JitDraw<false> {
    float nl, us;
};

template <bool PLAIN>
__device__ __forceinline__ JitDraw<PLAIN> jit_draw(uint32_t e, uint32_t traj, uint32_t m, const SsaParams &p,
                                                   const uint64_t *ltab)
{
    uint32_t w0, w1, w2, w3;
    philox10(e, traj, m, 0u, p.rk0, p.rk1, w0, w1, w2, w3);
    JitDraw<PLAIN> d;
    if constexpr (PLAIN) {
        fp64i_neglog53_norm(odd53(w0, w1), ltab, d.sm, d.lz);  // -ln u01_52(w0, w1)
        d.us = u01_52(w2, w3);
    } else {
        d.nl = -__logf(u01_23(w0));
        d.us = u01_23(w2);
    }
    return d;
}

// tau = -ln(u_tau) / a_0 (Eq. 2a), widened to FP64: FP64 path rounded once
// from the fixed-point logarithm (fp64i_tau, within 0.51 ulp), mixed path in
// FP32.
template <bool PLAIN>
__device__ __forceinline__ double jit_tau(const JitDraw<PLAIN> &d, typename Prec<PLAIN>::T a0)
{
    if constexpr (PLAIN) return fp64i_tau(d.sm, d.lz, a0);
    else return f32_to_f64(__fdividef(d.nl, a0));
}

// r = u_sel a_0 (Eq. 2b) rounded once, in the path's precision.  (The FP64
// product stays on the FP64 pipe: its integer form costs about 55 issue
// slots, more than the pipe time it frees.)
template <bool PLAIN>
__device__ __forceinline__ typename Prec<PLAIN>::T jit_sel_target(const JitDraw<PLAIN> &d,
                                                                  typename Prec<PLAIN>::T a0)
{
    if constexpr (PLAIN) return __dmul_rn(d.us, a0);
    else return __fmul_rn(d.us, a0);
}

#ifndef JIT_MEDIUM
// One warp's scratch for the cooperative tail: the trajectory's committed
// state, written by its owner before and read back after.
struct JitCoopState {
    double t;
    uint32_t e, pad;
    int32_t x[JS];
};
static_assert(sizeof(JitCoopState) <= SMC_JIT_COOP_BYTES, "cooperative scratch");

// The cooperative tail (see above): rounds of speculation until an event the
// full sequence has to handle (the owner then takes it); out of line, so its
// registers do not weigh on the event loop.
template <bool PLAIN>
__device__ __noinline__ void jit_coop(const SsaParams &p, const MonProg &P, const uint64_t *ltab, const int m,
                                      const uint32_t traj, const long long hb, const uint32_t ab0,
                                      const bool snapped, JitCoopState *st, const int lane)
{
    typedef typename Prec<PLAIN>::T T;
    const uint32_t *blob = p.blobs + p.blob_off[m];
    const T *cg = reinterpret_cast<const T *>(blob + blob[PLAIN ? BH_RATE_D : BH_RATE_F]);
    T c[JR];
#pragma unroll
    for (int k = 0; k < JR; ++k) c[k] = cg[k];
    const bool unbounded = P.unbounded != 0;
    const double t_max = P.t_max;
    const uint64_t budget = p.budget;
    const bool snap_open = p.snap_mode != 0 && !snapped;
    int32_t xb[JS];
#pragma unroll
    for (int i = 0; i < JS; ++i) xb[i] = st->x[i];
    double tb = st->t;
    uint32_t eb = st->e;
    // the lane's path: depth d and the reactions k1 (d >= 1), k2 (d = 2)
    int d = 0, k1 = 0, k2 = 0;
    if (lane >= 1 && lane <= JR) {
        d = 1;
        k1 = lane - 1;
    } else if (JIT_COOP_DEPTH == 2 && lane > JR && lane <= JR + JR * JR) {
        d = 2;
        k1 = (lane - 1 - JR) / JR;
        k2 = (lane - 1 - JR) % JR;
    }
    for (bool go = true; go;) {
        int32_t xs[JS];
#pragma unroll
        for (int i = 0; i < JS; ++i) xs[i] = xb[i];
        if (d >= 1) jit_apply(k1, xs, 1);
        if (d == 2) jit_apply(k2, xs, 1);
        T pre[JR];
        uint32_t pos = 0;
        if constexpr (PLAIN) jit_props_plain(xs, c, pre, pos);
        else jit_props_mixed(xs, c, pre, pos);
        const T a0 = pre[JR - 1];
        const bool dead = PLAIN ? __double_as_longlong((double)a0) <= 0 : !(a0 > (T)0);
        const JitDraw<PLAIN> dr = jit_draw<PLAIN>(eb + (uint32_t)d, traj, (uint32_t)m, p, ltab);
        const double tau = jit_tau<PLAIN>(dr, a0);  // the clock step, widened to FP64
        const T r = jit_sel_target<PLAIN>(dr, a0);
        int j = -1;
#pragma unroll
        for (int k = JR - 1; k >= 0; --k) {
            const bool hit = PLAIN ? __double_as_longlong((double)pre[k]) > __double_as_longlong((double)r)
                                   : pre[k] > r;
            if (hit) j = k;
        }
        if (j < 0) j = dead ? 0 : 31 - __clz(pos);
        jit_apply(j, xs, 1);
        const uint32_t abn = jit_atoms(xs);
        // walk the realized path: lane 0, then 1 + j0, then 1 + JR + j0 JR + j1
        int src = 0;
#pragma unroll
        for (int level = 0; level <= JIT_COOP_DEPTH; ++level) {
            const int jr = __shfl_sync(FULL_MASK, j, src);
            const double taur = __shfl_sync(FULL_MASK, tau, src);
            const bool deadr = __shfl_sync(FULL_MASK, (int)dead, src) != 0;
            const uint32_t abr = __shfl_sync(FULL_MASK, abn, src);
            const double tn = __dadd_rn(tb, taur);
            const bool rare = deadr | (__double_as_longlong(tn) > hb) | (abr != ab0) |
                              ((uint64_t)eb + 1u >= budget) | (snap_open & dgt(tn, p.t_snap)) |
                              (unbounded & dgt(tn, t_max));
            if (rare) {  // the owner takes this event through the full sequence
                go = false;
                break;
            }
            jit_apply(jr, xb, 1);
            tb = tn;
            ++eb;
            src = level == 0 ? 1 + jr : 1 + JR + (src - 1) * JR + jr;
        }
    }
    __syncwarp();
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < JS; ++i) st->x[i] = xb[i];
        st->t = tb;
        st->e = eb;
    }
}
#endif

template <bool PLAIN>
__device__ __forceinline__ void jit_run_instance(const SsaParams &p, const MonProg &P, const uint64_t *ltab,
                                                 const int m, double *tc, typename Prec<PLAIN>::T *crate,
                                                 const uint32_t *sdelta, void *coop, const int lane)
{
#ifndef JIT_MEDIUM
    JitCoopState *scratch = reinterpret_cast<JitCoopState *>(coop);
#else
    (void)coop;
#endif
    typedef typename Prec<PLAIN>::T T;
    const uint32_t *blob = p.blobs + p.blob_off[m];
#ifdef JIT_MEDIUM
    T *c = crate;  // the instance's rates in the warp's shared-memory slice
    {
        const T *rg = reinterpret_cast<const T *>(blob + blob[PLAIN ? BH_RATE_D : BH_RATE_F]);
        for (int k = lane; k < JR; k += 32) c[k] = rg[k];
        __syncwarp();
    }
#else
    (void)crate;
    (void)sdelta;
    T c[JR];
    if constexpr (PLAIN) {
        const double *rd = reinterpret_cast<const double *>(blob + blob[BH_RATE_D]);
#pragma unroll
        for (int k = 0; k < JR; ++k) c[k] = rd[k];
    } else {
        const float *rf = reinterpret_cast<const float *>(blob + blob[BH_RATE_F]);
#pragma unroll
        for (int k = 0; k < JR; ++k) c[k] = rf[k];
    }
#endif
    const int32_t *x0 = reinterpret_cast<const int32_t *>(blob + blob[BH_X0]);
    const unsigned long long tend = p.uniform ? p.u_end : p.tend[m];
    const bool always_step = P.has_lower != 0;
    const bool unbounded = P.unbounded != 0;
    const double t_max = P.t_max;
    const uint64_t budget = p.budget;
    const int snap_mode = p.snap_mode;
    const double t_snap = p.t_snap;

    bool active = false, exhausted = false, snapped = false;
    uint32_t traj = 0, e = 0;
    double t = 0.0;
    int32_t x[JS];
    JitDraw<PLAIN> nd;  // the current event's random numbers
    MonLane ml;
    MonHot mh;
    uint32_t c_yes = 0, c_dec = 0, c_bud = 0;
    // The common event's test folded into two numbers: hbe, the bit pattern
    // above which a clock must go through the full sequence (the monitor's
    // horizon, the snapshot time while it is open, t_max for the pessimistic
    // rule; -1 while the monitor sees every draw), and the event count from
    // which the budget stops a trajectory.
    long long hbe = -1;
    const uint32_t elim = budget == 0u ? 0u : (budget - 1u >= 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)(budget - 1u));
    const long long snap_bits = __double_as_longlong(t_snap), tmax_bits = __double_as_longlong(t_max);
    auto horizon = [&]() {
        long long h = mh.hb;
        if (snap_mode && !snapped) h = snap_bits < h ? snap_bits : h;
        if (unbounded) h = tmax_bits < h ? tmax_bits : h;
        hbe = (always_step || mh.pend) ? -1ll : h;
    };
    unsigned long long c_ev = 0;

    // verdict codes: 1 false, 2 true, 3 event budget exhausted, 4 stopped at
    // the snapshot (prefix-only run: no verdict, not counted)
    auto finish = [&](int v) {
        if (v == 3) ++c_bud;
        else if (v != 4) { ++c_dec; c_yes += (v == 2); }
        c_ev += e;
        const uint64_t idx = (uint64_t)m * p.out_stride + ((uint64_t)traj - p.out_base);
        if (p.o_verdict) {
            p.o_verdict[idx] = (v == 2);
            if (p.o_status) p.o_status[idx] = (v == 3) ? 1 : (v == 4 ? 2 : 0);
            if (p.o_events) p.o_events[idx] = e;
            if (p.o_tfinal) p.o_tfinal[idx] = t;
            if (p.o_xfinal) {
#pragma unroll
                for (int i = 0; i < JS; ++i) p.o_xfinal[idx * p.x_stride + i] = x[i];
            }
        }
        if (snap_mode && !snapped) {  // decided before t_snap
            p.o_snap[idx] = 1;
            if (p.o_esnap) p.o_esnap[idx] = e;
        }
        active = false;
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
                        traj = (uint32_t)id;
                        e = 0;
                        t = 0.0;
                        snapped = false;
#pragma unroll
                        for (int i = 0; i < JS; ++i) x[i] = x0[i];
                        nd = jit_draw<PLAIN>(0u, traj, (uint32_t)m, p, ltab);
                        ml.ab = jit_atoms(x);
                        mon_start(ml, P);
                        active = true;
                        const int v = mon_state(ml, P, 0.0, tc);
                        mh.load(ml);
                        horizon();
                        if (v) finish(v);
                    }
                }
                act = __ballot_sync(FULL_MASK, active);
            }
        }
        if (!act) {
            if (exhausted) break;
            continue;
        }
#ifndef JIT_MEDIUM
        // FP64 path only: on the mixed path the out-of-line call's register
        // saves cost the event loop more throughput than the tail gains
        // (measured: 52.6M -> 49.3M trajectories/s on Lotka-Volterra)
        if constexpr (PLAIN) if (exhausted && __popc(act) == 1 && !always_step) {
            const int owner = __ffs(act) - 1;
            // (not while the monitor looks at every draw: pending units, or a
            // clock already past the horizon of its windows)
            const bool quiet = mh.pend == 0u && __double_as_longlong(t) <= mh.hb;
            if (__shfl_sync(FULL_MASK, (int)quiet, owner) != 0) {
                // the owner's state goes through the warp's scratch (the
                // monitor's state stays with the owner: speculation stops at
                // the first event it has to look at)
                if (lane == owner) {
#pragma unroll
                    for (int i = 0; i < JS; ++i) scratch->x[i] = x[i];
                    scratch->t = t;
                    scratch->e = e;
                }
                __syncwarp();
                jit_coop<PLAIN>(p, P, ltab, m, __shfl_sync(FULL_MASK, traj, owner),
                                __shfl_sync(FULL_MASK, mh.hb, owner), __shfl_sync(FULL_MASK, mh.ab, owner),
                                __shfl_sync(FULL_MASK, (int)snapped, owner) != 0, scratch, lane);
                __syncwarp();
                if (lane == owner) {
#pragma unroll
                    for (int i = 0; i < JS; ++i) x[i] = scratch->x[i];
                    t = scratch->t;
                    e = scratch->e;
                    nd = jit_draw<PLAIN>(e, traj, (uint32_t)m, p, ltab);
                }
            }
        }
#endif
        if (!active) continue;

        // ---- one event (Sec. 2.2 steps 1-5) ----------------------------------
        // Small networks: everything an ordinary event needs is computed
        // without a branch (propensities, clock, selection, the next event's
        // draw, x += v_j, atoms); one test then sends the rare events
        // (absorbing state, snapshot, the monitor's clock window or atoms,
        // the event budget) through the full sequence, with x restored first.
        T pre[JR];
        uint32_t pos = 0;
        if constexpr (PLAIN) jit_props_plain(x, c, pre, pos);
        else jit_props_mixed(x, c, pre, pos);
        const T a0 = pre[JR - 1];
        const bool dead = PLAIN ? __double_as_longlong((double)a0) <= 0 : !(a0 > (T)0);
        const double tn = __dadd_rn(t, jit_tau<PLAIN>(nd, a0));
        const T r = jit_sel_target<PLAIN>(nd, a0);
        // step 2: the first j whose running sum exceeds r
        int j = -1;
#pragma unroll
        for (int k = JR - 1; k >= 0; --k) {
            const bool hit = PLAIN ? __double_as_longlong((double)pre[k]) > __double_as_longlong((double)r)
                                   : pre[k] > r;
            if (hit) j = k;
        }
        if (j < 0) {  // r reached the full sum (rounding): the last positive a_k, recomputed here
            T pre2[JR];
            uint32_t pos2 = 0;
            if constexpr (PLAIN) jit_props_plain(x, c, pre2, pos2);
            else jit_props_mixed(x, c, pre2, pos2);
            j = dead ? 0 : 31 - __clz(pos2);
        }
        const JitDraw<PLAIN> nd_next = jit_draw<PLAIN>(e + 1u, traj, (uint32_t)m, p, ltab);
#ifndef JIT_MEDIUM
        // step 4: x += v_j, then the common case: nothing for the monitor,
        // no snapshot, no stop (medium networks measured faster without it)
        jit_apply(j, x, 1);
        {
            const uint32_t abn = jit_atoms(x);
            const bool rare = dead | (__double_as_longlong(tn) > hbe) | (abn != mh.ab) | (e >= elim);
            if (!rare) {
                ++e;
                t = tn;
                nd = nd_next;
                continue;
            }
        }
        jit_apply(j, x, -1);
#endif
        if (dead) {
            finish(mon_close(ml, P));  // absorbing state: no further position
            continue;
        }
        nd = nd_next;
        if (snap_mode && !snapped && dgt(tn, t_snap)) {
            snapped = true;
            horizon();
            const uint64_t idx = (uint64_t)m * p.out_stride + ((uint64_t)traj - p.out_base);
            p.o_snap[idx] = 0;
            if (p.o_esnap) p.o_esnap[idx] = e;
#pragma unroll
            for (int i = 0; i < JS; ++i) p.o_xsnap[idx * p.x_stride + i] = x[i];
            if (snap_mode == 2) { finish(4); continue; }
        }
        int v = 0;
        if (mh.pend || __double_as_longlong(tn) > mh.hb) {
            v = mon_draw(ml, P, tn, tc);
            mh.load(ml);
            horizon();
        }
        if (!v && unbounded && dgt(tn, t_max)) v = 1;  // pessimistic rule (Sec. 3.2)
        if (v) { finish(v); continue; }

        // step 4: x += v_j, then the monitor at the new state
#ifdef JIT_MEDIUM
        jit_apply_row(sdelta + j * JW, x, 1);
#else
        jit_apply(j, x, 1);
#endif
        ++e;
        t = tn;
        const uint32_t ab = jit_atoms(x);
        if (always_step || ab != mh.ab || mh.pend) {
            ml.ab = ab;
            v = mon_state(ml, P, t, tc);
            mh.load(ml);
            horizon();
        }
        if (v) finish(v);
        else if ((uint64_t)e >= budget) finish(3);
    }

    const unsigned long long s_yes = warp_sum(c_yes), s_dec = warp_sum(c_dec);
    const unsigned long long s_ev = warp_sum(c_ev), s_bud = warp_sum(c_bud);
    if (lane == 0 && (s_dec | s_bud)) {
        atomicAdd(&p.counts[4 * m + 0], s_yes);
        atomicAdd(&p.counts[4 * m + 1], s_dec);
        atomicAdd(&p.counts[4 * m + 2], s_ev);
        atomicAdd(&p.counts[4 * m + 3], s_bud);
    }
}

template <bool PLAIN>
__device__ __forceinline__ void jit_kernel_body(const SsaParams &p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_last;
    stage_block_tables(p, smem, PLAIN);
    const MonProg &P = *reinterpret_cast<const MonProg *>(smem);
    const uint64_t *ltab = reinterpret_cast<const uint64_t *>(smem + sizeof(MonProg));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // block: monitor program | logarithm table (FP64 path) | net-change table
    // (medium networks) | warp slices
    uint32_t *sdelta = reinterpret_cast<uint32_t *>(smem + sizeof(MonProg) + p.logtab_bytes);
#ifdef JIT_MEDIUM
    for (int i = threadIdx.x; i < JR * JW; i += blockDim.x) sdelta[i] = kJitDelta[i];
    __syncthreads();
#endif
    // warp slice: the nested operators' candidate clocks tc[units][32], then
    // (medium networks) the current instance's rates
    unsigned char *ws = smem + sizeof(MonProg) + p.logtab_bytes + JIT_DELTA_BYTES + (size_t)warp * p.warp_bytes;
    double *tc = reinterpret_cast<double *>(ws) + lane;
    typedef typename Prec<PLAIN>::T T;
    T *crate = reinterpret_cast<T *>(ws + p.tc_bytes);
    void *coop = ws + p.warp_bytes - SMC_JIT_COOP_BYTES;  // the cooperative tail's scratch (small networks)
    bool first = true;
    const int gw = blockIdx.x * (blockDim.x >> 5) + warp;
    for (;;) {
        const int m = acquire_instance(p, first, gw, lane);
        if (m < 0) break;
        jit_run_instance<PLAIN>(p, P, ltab, m, tc, crate, sdelta, coop, lane);
        __syncwarp();
    }
    wilson_epilogue(p, &s_last);
}

}  // namespace

extern "C" __global__ void __launch_bounds__(256, JIT_MINB_PLAIN) smc_jit_ssa_plain(const SsaParams p)
{
    jit_kernel_body<true>(p);
}

extern "C" __global__ void __launch_bounds__(256, JIT_MINB_MIXED) smc_jit_ssa_mixed(const SsaParams p)
{
    jit_kernel_body<false>(p);
}
