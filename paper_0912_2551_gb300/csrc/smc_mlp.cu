// smc_mlp.cu -- the surrogate network used as a control variate: forward,
// backward and Adam update as hand-written BF16 tensor-core kernels with
// FP32 accumulation and FP32 master weights.  Every product runs on tcgen05
// (operands in shared memory, accumulators in tensor memory): inference on
// the estimator's path, and the training step's forward pass, backward pass
// and weight gradients (smc_mlp_train.cuh).
//
// Network: g(x) = sigmoid(w4 . h3 + b4), h_l = relu(W_l h_{l-1} + b_l),
// x in R^16 (zero-padded features), hidden width 128.  Training minimises the
// binary cross-entropy of g against the trajectory verdicts.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <random>
#include <string>
#include <vector>

#include "smc.h"
#include "smc_mlp.h"
#include "smc_tc.h"

typedef __nv_bfloat16 bf16;

namespace {

constexpr int H = MLP_H, IN = MLP_IN;

__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ float2 unpack2(uint32_t w)
{
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w));
}

// ---------------------------------------------------------------------------
// Inference on the fifth-generation tensor cores (tcgen05).  A CTA runs
// kTcGroups independent pipelines of 128 threads; each pipeline works on one
// 128-row tile at a time with its layer accumulator (128 rows x 128 FP32
// columns) in its own quarter of the SM's tensor memory.  The weights are
// staged once per CTA and shared; while one pipeline runs its epilogue on
// the CUDA cores, the others' MMAs keep the tensor cores busy.
//
// Operands in shared memory use the K-major core-matrix layout without
// swizzling of smc_tc.h (8-row x 16-byte core matrices of 128 contiguous
// bytes); one MMA consumes K = 16, i.e. two core matrices along K: step s
// starts 256 * s bytes into the operand.
//
// Everything but the ReLU runs on the tensor cores.  Each layer's
// accumulator starts as its bias: an MMA of a constant tile of ones (A,
// columns 0 and 1) with a bias tile (B, columns 0 and 1 = the FP32 bias
// split into BF16 high and low parts, b = hi + lo to about 2^-17).  The
// output unit is an N = 16 MMA whose B rows 0 and 1 are w4's high and low
// parts, so z = D[:, 0] + D[:, 1].
//
// Per tile: features -> X (K = 16, in the first 4 KB of the activation
// buffer); bias + MMA (W1); epilogue: tensor memory -> registers (thread i
// of the pipeline holds row i, the accumulator's lane i), ReLU and BF16 in
// one conversion, back to shared memory as the next layer's A operand;
// bias + MMAs (W2, K = 128), epilogue; bias + MMAs (W3), epilogue; bias +
// MMAs (w4, N = 16); g = 1 / (1 + e^-z).  The pipeline's first thread
// issues the MMAs and commits them to the pipeline's mbarrier, which its
// 128 threads wait on.
// ---------------------------------------------------------------------------

constexpr int kTcRows = 128;                    // rows per tile = TMEM lanes
constexpr int kTcGroups = 4;                    // pipelines per CTA
constexpr int kTcThreads = 128 * kTcGroups;
constexpr int kTcSmW1 = 0;                      // W1 [128][16]  BF16, 4 KB
constexpr int kTcSmW2 = kTcSmW1 + H * IN * 2;   // W2 [128][128] BF16, 32 KB
constexpr int kTcSmW3 = kTcSmW2 + H * H * 2;    // W3 [128][128] BF16, 32 KB
constexpr int kTcSmW4 = kTcSmW3 + H * H * 2;    // [16][128]: w4 high, w4 low, zeros; 4 KB
constexpr int kTcSmOnes = kTcSmW4 + 16 * H * 2; // [128][16]: ones in columns 0, 1; 4 KB
constexpr int kTcSmB1 = kTcSmOnes + kTcRows * 16 * 2;  // bias tiles [128][16], 4 KB each (layers 1-3)
constexpr int kTcSmB4 = kTcSmB1 + 3 * H * 16 * 2;      // [16][16]: b4 high, low in row 0
constexpr int kTcSmBar = kTcSmB4 + 16 * 16 * 2;        // one mbarrier per pipeline, the weights' mbarrier, the TMEM address
constexpr int kTcSmGroup = (kTcSmBar + 8 * (kTcGroups + 1) + 4 + 1023) / 1024 * 1024;
constexpr int kTcGroupBytes = kTcRows * H * 2;  // activations [128][128] (features [128][16] at the start)
constexpr int kTcSmem = kTcSmGroup + kTcGroups * kTcGroupBytes;
constexpr uint32_t kTcCols = 128 * kTcGroups;   // TMEM columns per CTA: all 512 of the SM
constexpr uint32_t kTcWaitLimit = 1u << 26;     // mbarrier polls before a wait gives up
constexpr uint64_t kTcWaitNs = 1000000000ull;   // or this much wall time (1 s)
static_assert(kTcSmBar % 8 == 0, "mbarrier alignment");
static_assert(kTcSmem <= 227 * 1024, "shared memory per CTA");
// the CTA takes the whole tensor memory, so two must never share an SM
static_assert(2 * (kTcSmem + 1024) > 228 * 1024, "one CTA per SM");

__host__ __device__ constexpr uint32_t tc_idesc(int N) { return tc_idesc_bf16(kTcRows, N); }

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// barrier over one pipeline's 128 threads (named barrier id, 1..kTcGroups)
__device__ __forceinline__ void group_sync(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }

// the same barrier, returning whether v was true in any of the 128 threads
__device__ __forceinline__ bool group_or(int id, bool v)
{
    uint32_t r;
    asm volatile(
        "{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n bar.red.or.pred po, %2, 128, pi;\n"
        " selp.u32 %0, 1, 0, po;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id)
        : "memory");
    return r != 0;
}

// waits for the mbarrier's phase `parity` to complete; false once about
// kTcWaitNs of wall time (global timer) or kTcWaitLimit polls have passed
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity)
{
    uint64_t t0 = 0;
    for (uint32_t i = 0; i < kTcWaitLimit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((i & 63) == 0) {
            uint64_t t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            if (i == 0) t0 = t;
            else if (t - t0 > kTcWaitNs) return false;
        }
    }
    return false;
}

// starts loading 32 consecutive FP32 columns of this thread's accumulator
// lane; the registers hold them only after tc_wait_ld(r)
__device__ __forceinline__ void tc_load32_async(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}

// waits for this thread's outstanding tensor-memory loads; naming r as
// read-write keeps the compiler from using r before the wait
__device__ __forceinline__ void tc_wait_ld(uint32_t (&r)[32])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;\n"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

// two consecutive FP32 columns of this thread's accumulator lane
__device__ __forceinline__ void tc_load2(uint32_t taddr, uint32_t (&r)[2])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1])
        : "r"(taddr)
        : "memory");
}

// relu, rounded to BF16 and packed: lo in the low half (first in memory)
__device__ __forceinline__ uint32_t relu_pack2(uint32_t lo, uint32_t hi)
{
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(__uint_as_float(hi)), "f"(__uint_as_float(lo)));
    return d;
}

// The BF16 weights live in global memory already in the K-major
// core-matrix layout (the update kernel writes them so): W1 [128][16],
// 4 KB, then W2 and W3 [128][128], 32 KB each.  A kernel stages all three
// into shared memory (W1, W2, W3 contiguous from byte w_off) with bulk
// copies completing on one mbarrier; issued by one thread after the
// mbarrier's initialisation.
constexpr uint32_t kW1Bytes = H * IN * 2, kWHBytes = H * H * 2, kWBytes = kW1Bytes + 2 * kWHBytes;

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void stage_weights(uint32_t w_off, const bf16 *w1b, const bf16 *w2b, const bf16 *w3b,
                                              uint32_t bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kWBytes) : "memory");
    bulk_g2s(w_off, w1b, kW1Bytes, bar);
    bulk_g2s(w_off + kW1Bytes, w2b, kWHBytes, bar);
    bulk_g2s(w_off + kW1Bytes + kWHBytes, w3b, kWHBytes, bar);
}

__device__ __forceinline__ uint32_t pack_bf16x2(bf16 lo, bf16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// element (r, k) of an operand with K columns in the core-matrix layout
__device__ __forceinline__ bf16 *tc_elem(unsigned char *base, int r, int k, int K)
{
    return reinterpret_cast<bf16 *>(base + tc_elem_offset(r, k, K));
}

// high and low BF16 parts of an FP32 value (v = hi + lo to about 2^-17 relative)
__device__ __forceinline__ bf16 bf16_hi(float v) { return __float2bfloat16_rn(v); }
__device__ __forceinline__ bf16 bf16_lo(float v) { return __float2bfloat16_rn(v - __bfloat162float(__float2bfloat16_rn(v))); }

// The forward pass over n rows, one persistent launch (one CTA of
// kTcThreads per SM) over 128-row tiles, weights staged once per CTA.
// FP32 features x [n][n_in] (n_in <= 16), rounded to BF16 as the training
// input is; g[r] = 1 / (1 + e^-z); rows with skip[r] != 0 (skip may be
// null) need no output, and a tile whose rows all skip is not computed.  A
// wait that gives up sets *err and leaves NaN in the outputs of the tile it
// was working on, and that pipeline stops.
__global__ void __launch_bounds__(kTcThreads) mlp_tc_forward(const float *__restrict__ x, uint64_t n, int n_in,
                                                             const uint8_t *__restrict__ skip, const bf16 *w1b,
                                                             const bf16 *w2b, const bf16 *w3b, const float *master,
                                                             float *g_out, int *err)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + kTcSmBar);
    const uint32_t bar_w = smem_u32(bars + kTcGroups);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + kTcSmBar + 8 * (kTcGroups + 1));
    const int tid = threadIdx.x, warp = tid >> 5, grp = tid >> 7, gt = tid & 127;
    const int bid = 1 + grp;  // the pipeline's named barrier

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i <= kTcGroups; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bars + i)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        stage_weights(smem_u32(sm + kTcSmW1), w1b, w2b, w3b, bar_w);
    }
    const bf16 zero = __float2bfloat16_rn(0.0f), one = __float2bfloat16_rn(1.0f);
    if (tid < H) {  // thread r: row r of the ones and bias tiles, column r of the output unit's tile
        const int r = tid;
        const float bl[3] = {master[MLP_OFF_B1 + r], master[MLP_OFF_B2 + r], master[MLP_OFF_B3 + r]};
        const float w = master[MLP_OFF_W4 + r], b4 = master[MLP_OFF_B4];
        const uint4 z4 = make_uint4(0u, 0u, 0u, 0u);
        auto row16 = [&](int off, bf16 v0, bf16 v1) {  // columns 0, 1 = v0, v1; 2-15 zero
            *reinterpret_cast<uint4 *>(sm + off + tc_core_offset(r, 0, 16)) = make_uint4(pack_bf16x2(v0, v1), 0u, 0u, 0u);
            *reinterpret_cast<uint4 *>(sm + off + tc_core_offset(r, 1, 16)) = z4;
        };
        row16(kTcSmOnes, one, one);
#pragma unroll
        for (int l = 0; l < 3; ++l) row16(kTcSmB1 + l * H * 16 * 2, bf16_hi(bl[l]), bf16_lo(bl[l]));
#pragma unroll
        for (int j = 0; j < 16; ++j)  // output unit: rows 0, 1 = w4 high, low
            *tc_elem(sm + kTcSmW4, j, r, H) = j == 0 ? bf16_hi(w) : j == 1 ? bf16_lo(w) : zero;
        if (r < 16) {  // [16][16]: b4 high, low in row 0
            const bf16 v0 = r == 0 ? bf16_hi(b4) : zero, v1 = r == 0 ? bf16_lo(b4) : zero;
            *reinterpret_cast<uint4 *>(sm + kTcSmB4 + tc_core_offset(r, 0, 16)) = make_uint4(pack_bf16x2(v0, v1), 0u, 0u, 0u);
            *reinterpret_cast<uint4 *>(sm + kTcSmB4 + tc_core_offset(r, 1, 16)) = z4;
        }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // the weights' copies (bounded wait; a CTA that gives up computes nothing)
    const bool w_failed = __syncthreads_or(!tc_wait(bar_w, 0));
    bool failed = w_failed;
    const uint32_t tmem = *tmem_slot;
    const uint32_t tacc = tmem + 128u * grp;                              // the pipeline's columns
    const uint32_t t_row = tacc + ((uint32_t)(32 * (warp & 3)) << 16);  // this warp's 32 lanes

    unsigned char *act = sm + kTcSmGroup + grp * kTcGroupBytes;
    const uint32_t bar = smem_u32(bars + grp);
    const uint32_t aAct = smem_u32(act), aOnes = smem_u32(sm + kTcSmOnes);
    uint32_t phase = 0;
    const uint64_t tiles = failed ? 0 : (n + kTcRows - 1) / kTcRows;

    // a tile's features and mask are loaded one tile ahead, so their
    // latency overlaps the previous tile's layers
    const uint64_t stride = (uint64_t)gridDim.x * kTcGroups;
    auto load_tile = [&](uint64_t t, float (&f)[IN], bool &nd) {
        const uint64_t r = t * kTcRows + gt;
        nd = r < n && !(skip && skip[r]);
#pragma unroll
        for (int k = 0; k < IN; ++k) f[k] = (r < n && k < n_in) ? x[r * n_in + k] : 0.0f;
    };
    float f_next[IN];
    bool need_next = false;
    uint64_t tile = (uint64_t)blockIdx.x * kTcGroups + grp;
    if (tile < tiles) load_tile(tile, f_next, need_next);
    for (; tile < tiles; tile += stride) {
        const uint64_t row = tile * kTcRows + gt;
        float f[IN];
#pragma unroll
        for (int k = 0; k < IN; ++k) f[k] = f_next[k];
        const bool need = need_next;
        if (tile + stride < tiles) load_tile(tile + stride, f_next, need_next);
        if (!group_or(bid, need)) continue;
        {   // features -> X (zero-padded to 16, BF16)
#pragma unroll
            for (int kg = 0; kg < IN / 8; ++kg) {
                uint4 v;
                v.x = pack2(f[8 * kg], f[8 * kg + 1]);
                v.y = pack2(f[8 * kg + 2], f[8 * kg + 3]);
                v.z = pack2(f[8 * kg + 4], f[8 * kg + 5]);
                v.w = pack2(f[8 * kg + 6], f[8 * kg + 7]);
                *reinterpret_cast<uint4 *>(act + tc_core_offset(gt, kg, IN)) = v;
            }
        }
        uint32_t zc[2] = {0u, 0u};
        for (int layer = 0; layer < 4; ++layer) {
            // operands written by every thread -> visible to the tensor core;
            // the previous epilogue's tensor-memory reads are complete
            fence_async_smem();
            tc_fence_before();
            group_sync(bid);
            if (gt == 0) {
                tc_fence_after();
                if (layer == 0) {
                    tc_mma(tacc, tc_desc(aOnes, kTcLbo, tc_sbo(16)),
                           tc_desc(smem_u32(sm + kTcSmB1), kTcLbo, tc_sbo(16)), tc_idesc(H), 0);
                    tc_mma(tacc, tc_desc(aAct, kTcLbo, tc_sbo(IN)), tc_desc(smem_u32(sm + kTcSmW1), kTcLbo, tc_sbo(IN)),
                           tc_idesc(H), 1);
                } else {
                    const int N = layer == 3 ? 16 : H;
                    const uint32_t aB = smem_u32(sm + (layer == 3 ? kTcSmB4 : kTcSmB1 + layer * H * 16 * 2));
                    const uint32_t aW = smem_u32(sm + (layer == 1 ? kTcSmW2 : layer == 2 ? kTcSmW3 : kTcSmW4));
                    tc_mma(tacc, tc_desc(aOnes, kTcLbo, tc_sbo(16)), tc_desc(aB, kTcLbo, tc_sbo(16)), tc_idesc(N), 0);
#pragma unroll
                    for (int s = 0; s < H / 16; ++s)
                        tc_mma(tacc, tc_desc(aAct + 256 * s, kTcLbo, tc_sbo(H)), tc_desc(aW + 256 * s, kTcLbo, tc_sbo(H)),
                               tc_idesc(N), 1);
                }
                tc_commit(bar);
            }
            const bool ok = tc_wait(bar, phase);
            phase ^= 1;
            if (group_or(bid, !ok)) {
                failed = true;
                break;
            }
            tc_fence_after();
            if (layer == 3) {
                tc_load2(t_row, zc);
                break;
            }
            {   // 4 chunks of 32 columns; the next chunk loads while this one converts
                uint32_t va[32], vb[32];
                auto store_chunk = [&](int c, const uint32_t (&v)[32]) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const uint4 w =
                            make_uint4(relu_pack2(v[8 * q], v[8 * q + 1]), relu_pack2(v[8 * q + 2], v[8 * q + 3]),
                                       relu_pack2(v[8 * q + 4], v[8 * q + 5]), relu_pack2(v[8 * q + 6], v[8 * q + 7]));
                        *reinterpret_cast<uint4 *>(act + tc_core_offset(gt, 4 * c + q, H)) = w;
                    }
                };
                tc_load32_async(t_row, va);
                tc_wait_ld(va);
                tc_load32_async(t_row + 32, vb);
                store_chunk(0, va);
                tc_wait_ld(vb);
                tc_load32_async(t_row + 64, va);
                store_chunk(1, vb);
                tc_wait_ld(va);
                tc_load32_async(t_row + 96, vb);
                store_chunk(2, va);
                tc_wait_ld(vb);
                store_chunk(3, vb);
            }
        }
        if (failed) {
            if (row < n) g_out[row] = __int_as_float(0x7fc00000);
            if (gt == 0) atomicExch(err, 1);
            break;
        }
        const float z = __uint_as_float(zc[0]) + __uint_as_float(zc[1]);
        if (need) g_out[row] = 1.0f / (1.0f + expf(-z));
    }
    // Release tensor memory once every MMA and load of this CTA has finished.
    // A pipeline that gave up waits again (bounded) for the completion of its
    // last committed MMAs: up to four more periods of kTcWaitNs.  Only if the
    // tensor cores never report it does the CTA release the memory without
    // the confirmation (a CTA may not exit holding tensor memory), and it
    // records that case (err = 2) for the host.
    if (w_failed) {  // no products were issued; the copies must land before the CTA exits
        if (tid == 0) {
            atomicExch(err, 1);
            bool drained = false;
            for (int k = 0; k < 4 && !drained; ++k) drained = tc_wait(bar_w, 0);
            if (!drained) atomicExch(err, 2);
        }
    } else if (failed && gt == 0) {
        bool drained = false;
        for (int k = 0; k < 4 && !drained; ++k) drained = tc_wait(bar, phase ^ 1);
        if (!drained) atomicExch(err, 2);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
    }
}

#include "smc_mlp_train.cuh"

// Sums the partial gradients (one per CTA of the training-step kernel,
// kPartStride floats apart), optionally applies Adam (lr > 0) to the FP32
// master weights, and refreshes their BF16 copies (in the K-major operand
// layout, which the kernels copy into shared memory as they are and read
// MN-major where they need the transpose).  Four threads per parameter:
// thread j of the four sums the partials j, j + 4, ... in order, and the
// four sums are added in a fixed order (deterministic).  ctr[0] is the
// sampling step (advanced here when lr > 0), ctr[1] Adam's step count t
// (advanced by the training-step kernel before this launch).
constexpr int kUpdThreads = 256, kUpdParams = kUpdThreads / 4;
__global__ void __launch_bounds__(kUpdThreads) mlp_update_kernel(int nparts, const float *part, float *master,
                                                                 float *am, float *av, float lr, float beta1,
                                                                 float beta2, float eps, unsigned long long *ctr,
                                                                 float *grad_out, bf16 *w1b, bf16 *w2b, bf16 *w3b)
{
    const int i = blockIdx.x * kUpdParams + (threadIdx.x >> 2), j = threadIdx.x & 3;
    if (lr > 0.0f && blockIdx.x == 0 && threadIdx.x == 0) ctr[0] += 1ull;
    float gsum = 0.0f;
    if (i < MLP_NPARAM) {
#pragma unroll 8
        for (int c = j; c < nparts; c += 4) gsum += part[(size_t)c * kPartStride + i];
    }
    gsum += __shfl_down_sync(0xffffffffu, gsum, 1, 4);  // (s0 + s1) + (s2 + s3) in lane j = 0
    gsum += __shfl_down_sync(0xffffffffu, gsum, 2, 4);
    if (i >= MLP_NPARAM || j != 0) return;
    if (grad_out) grad_out[i] = gsum;
    float w = master[i];
    if (lr > 0.0f) {
        const float t = (float)ctr[1];
        const float bc1 = 1.0f - powf(beta1, t), bc2 = 1.0f - powf(beta2, t);
        const float m = beta1 * am[i] + (1.0f - beta1) * gsum;
        const float v = beta2 * av[i] + (1.0f - beta2) * gsum * gsum;
        am[i] = m;
        av[i] = v;
        w -= lr * (m / bc1) / (sqrtf(v / bc2) + eps);
        master[i] = w;
    }
    const bf16 wb = __float2bfloat16(w);  // BF16 copies in the operand layout (rows = outputs, K = inputs)
    if (i < MLP_OFF_B1) {
        const int e = i - MLP_OFF_W1;
        w1b[tc_elem_offset(e / IN, e % IN, IN) / 2] = wb;
    } else if (i >= MLP_OFF_W2 && i < MLP_OFF_B2) {
        const int e = i - MLP_OFF_W2;
        w2b[tc_elem_offset(e / H, e % H, H) / 2] = wb;
    } else if (i >= MLP_OFF_W3 && i < MLP_OFF_B3) {
        const int e = i - MLP_OFF_W3;
        w3b[tc_elem_offset(e / H, e % H, H) / 2] = wb;
    }
}
constexpr int kUpdBlocks = (MLP_NPARAM + kUpdParams - 1) / kUpdParams;

constexpr int kMaxBatch = SMC_MLP_MAX_BATCH;  // rows per training step or gradient
constexpr int kMaxParts = 256;       // training-step CTAs (at most one per SM)
constexpr int kMaxEpochs = 4096;
constexpr int kGraphSteps = 32;      // training steps per captured graph

// The training steps of one smc_mlp_train call as CUDA graphs: `full` runs
// kGraphSteps steps, `rest` the remainder of an epoch; both read the step
// counters from device memory, so that one graph serves every launch.
struct TrainGraphs {
    cudaGraphExec_t full = nullptr, rest = nullptr;
    const float *x = nullptr, *y = nullptr;
    uint64_t n = 0, seed = 0;
    int batch = 0, n_full = 0, n_rest = 0;
    float lr = 0.0f;
};

}  // namespace

struct smc_mlp {
    int device = 0;
    int n_in = 0;
    int n_sm = 0;
    std::string err;
    cudaStream_t stream = nullptr;
    float *master = nullptr, *am = nullptr, *av = nullptr, *part = nullptr, *grad = nullptr;
    bf16 *w1b = nullptr, *w2b = nullptr, *w3b = nullptr;
    float *loss = nullptr;                  // per-epoch loss sums, then the running sum at [kMaxEpochs]
    unsigned long long *ctr = nullptr;      // sampling step, Adam's t
    int *h_err = nullptr, *d_err = nullptr; // a tensor-core wait gave up (mapped host memory)
    TrainGraphs graphs;
    cudaEvent_t graphs_done = nullptr;      // after the last launch of the cached graphs
};

namespace {

int mfail(smc_mlp *m, int code, const std::string &msg)
{
    if (m) m->err = msg;
    return code;
}

#define MCK(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return mfail(m, e_ == cudaErrorMemoryAllocation ? SMC_E_OOM : SMC_E_CUDA,              \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                      \
    } while (0)

int refresh(smc_mlp *m, cudaStream_t s)
{
    mlp_update_kernel<<<kUpdBlocks, kUpdThreads, 0, s>>>(0, m->part, m->master, m->am, m->av, 0.0f, 0.f,
                                                              0.f, 0.f, m->ctr, nullptr, m->w1b, m->w2b, m->w3b);
    MCK(cudaGetLastError());
    return SMC_OK;
}

// One training-step kernel over the rows of rs (loss sum added to
// *loss_acc; with adam, Adam's step count advanced); *nparts = the partial
// gradients it writes.  Tiles are spread evenly over at most one CTA per SM.
int step_launch(smc_mlp *m, const StepRows &rs, float *loss_acc, bool adam, cudaStream_t s, int *nparts)
{
    const int tiles = (rs.B + kTcRows - 1) / kTcRows;
    const int cap = std::min(m->n_sm, kMaxParts);
    const int per = (tiles + cap - 1) / cap;
    const int grid = (tiles + per - 1) / per;
    mlp_train_step_kernel<<<grid, kStThreads, kStSmem, s>>>(rs, 1.0f / (float)rs.B, m->w1b, m->w2b, m->w3b,
                                                             m->master, m->part, loss_acc,
                                                             adam ? m->ctr + 1 : nullptr, m->d_err);
    MCK(cudaGetLastError());
    *nparts = grid;
    return SMC_OK;
}

// k training steps (step kernel + Adam update each) on stream s
int enqueue_steps(smc_mlp *m, const StepRows &rs, float lr, int k, cudaStream_t s)
{
    for (int i = 0; i < k; ++i) {
        int parts = 0;
        const int rc = step_launch(m, rs, m->loss + kMaxEpochs, true, s, &parts);
        if (rc) return rc;
        mlp_update_kernel<<<kUpdBlocks, kUpdThreads, 0, s>>>(parts, m->part, m->master, m->am, m->av, lr,
                                                                  0.9f, 0.999f, 1e-8f, m->ctr, nullptr, m->w1b,
                                                                  m->w2b, m->w3b);
        MCK(cudaGetLastError());
    }
    return SMC_OK;
}

// captures k training steps into an executable graph (on the library's own
// stream, so that nothing else is captured)
int capture_steps(smc_mlp *m, const StepRows &rs, float lr, int k, cudaGraphExec_t *out)
{
    *out = nullptr;
    if (k == 0) return SMC_OK;
    MCK(cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal));
    const int rc = enqueue_steps(m, rs, lr, k, m->stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(m->stream, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    MCK(e);
    const cudaError_t ei = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    MCK(ei);
    return SMC_OK;
}

void drop_graphs(smc_mlp *m)
{
    if (m->graphs_done) cudaEventSynchronize(m->graphs_done);
    if (m->graphs.full) cudaGraphExecDestroy(m->graphs.full);
    if (m->graphs.rest) cudaGraphExecDestroy(m->graphs.rest);
    m->graphs = TrainGraphs{};
}

int check_waits(smc_mlp *m)
{
    if (*m->h_err)
        return mfail(m, SMC_E_CUDA, *m->h_err == 2 ? "a tensor-core wait gave up and tensor memory was released "
                                                      "without the completion of its products"
                                                    : "an earlier launch gave up waiting for the tensor cores");
    return SMC_OK;
}

}  // namespace

extern "C" {

int smc_mlp_create(smc_mlp **out, int device, int n_in, uint64_t seed)
{
    if (!out || n_in < 1 || n_in > MLP_IN) return SMC_E_INVALID_ARG;
    *out = nullptr;
    int nd = 0;
    if (cudaGetDeviceCount(&nd) != cudaSuccess || device < 0 || device >= nd) return SMC_E_NO_DEVICE;
    smc_mlp *m = new (std::nothrow) smc_mlp();
    if (!m) return SMC_E_OOM;
    m->device = device;
    m->n_in = n_in;
    auto fin = [&](int rc) {
        if (rc != SMC_OK) smc_mlp_destroy(m);
        else *out = m;
        return rc;
    };
    if (cudaSetDevice(device) != cudaSuccess) return fin(SMC_E_CUDA);
    if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess) return fin(SMC_E_CUDA);
    if (cudaEventCreateWithFlags(&m->graphs_done, cudaEventDisableTiming) != cudaSuccess) return fin(SMC_E_CUDA);
    const size_t np = MLP_NPARAM;
    void **f32[] = {(void **)&m->master, (void **)&m->am, (void **)&m->av, (void **)&m->grad};
    for (void **p : f32)
        if (cudaMalloc(p, np * 4) != cudaSuccess) return fin(SMC_E_OOM);
    if (cudaMalloc((void **)&m->part, (size_t)kMaxParts * kPartStride * 4) != cudaSuccess) return fin(SMC_E_OOM);
    void **wb[] = {(void **)&m->w1b, (void **)&m->w2b, (void **)&m->w3b};
    for (void **p : wb)
        if (cudaMalloc(p, (size_t)H * H * 2) != cudaSuccess) return fin(SMC_E_OOM);
    if (cudaMalloc((void **)&m->loss, (size_t)(kMaxEpochs + 1) * 4) != cudaSuccess) return fin(SMC_E_OOM);
    if (cudaMalloc((void **)&m->ctr, 2 * sizeof(unsigned long long)) != cudaSuccess) return fin(SMC_E_OOM);
    if (cudaMemset(m->ctr, 0, 2 * sizeof(unsigned long long)) != cudaSuccess) return fin(SMC_E_CUDA);
    if (cudaHostAlloc((void **)&m->h_err, sizeof(int), cudaHostAllocMapped) != cudaSuccess) return fin(SMC_E_OOM);
    *m->h_err = 0;
    if (cudaHostGetDevicePointer((void **)&m->d_err, m->h_err, 0) != cudaSuccess) return fin(SMC_E_CUDA);
    if (cudaDeviceGetAttribute(&m->n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return fin(SMC_E_CUDA);
    if (cudaFuncSetAttribute(mlp_tc_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem) != cudaSuccess ||
        cudaFuncSetAttribute(mlp_train_step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kStSmem) !=
            cudaSuccess)
        return fin(SMC_E_CUDA);
    // He-uniform initial weights from the seed; zero biases and Adam moments
    std::vector<float> w(np, 0.0f);
    std::mt19937_64 gen(seed);
    auto fill = [&](int off, int fan_out, int fan_in, int fan_used) {
        const float lim = std::sqrt(6.0f / (float)fan_used);
        std::uniform_real_distribution<float> U(-lim, lim);
        for (int o = 0; o < fan_out; ++o)
            for (int i = 0; i < fan_in; ++i) w[off + o * fan_in + i] = (i < fan_used) ? U(gen) : 0.0f;
    };
    fill(MLP_OFF_W1, H, IN, n_in);
    fill(MLP_OFF_W2, H, H, H);
    fill(MLP_OFF_W3, H, H, H);
    fill(MLP_OFF_W4, 1, H, H);
    if (cudaMemcpy(m->master, w.data(), np * 4, cudaMemcpyHostToDevice) != cudaSuccess) return fin(SMC_E_CUDA);
    if (cudaMemset(m->am, 0, np * 4) != cudaSuccess || cudaMemset(m->av, 0, np * 4) != cudaSuccess)
        return fin(SMC_E_CUDA);
    if (refresh(m, m->stream) != SMC_OK || cudaStreamSynchronize(m->stream) != cudaSuccess) return fin(SMC_E_CUDA);
    return fin(SMC_OK);
}

void smc_mlp_destroy(smc_mlp *m)
{
    if (!m) return;
    cudaSetDevice(m->device);
    if (m->stream) cudaStreamSynchronize(m->stream);
    drop_graphs(m);
    void *ptrs[] = {m->master, m->am, m->av, m->part, m->grad, m->w1b, m->w2b, m->w3b, m->loss, m->ctr};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (m->h_err) cudaFreeHost(m->h_err);
    if (m->graphs_done) cudaEventDestroy(m->graphs_done);
    if (m->stream) cudaStreamDestroy(m->stream);
    delete m;
}

const char *smc_mlp_last_error(const smc_mlp *m) { return m ? m->err.c_str() : ""; }

}  // extern "C"

int smc_mlp_inputs(const smc_mlp *m) { return m ? m->n_in : 0; }

extern "C" {

int smc_mlp_get_params(smc_mlp *m, float *host)
{
    if (!m || !host) return SMC_E_INVALID_ARG;
    MCK(cudaSetDevice(m->device));
    if (m->graphs_done) MCK(cudaEventSynchronize(m->graphs_done));
    MCK(cudaStreamSynchronize(m->stream));
    MCK(cudaMemcpy(host, m->master, (size_t)MLP_NPARAM * 4, cudaMemcpyDeviceToHost));
    return SMC_OK;
}

int smc_mlp_set_params(smc_mlp *m, const float *host)
{
    if (!m || !host) return SMC_E_INVALID_ARG;
    MCK(cudaSetDevice(m->device));
    if (m->graphs_done) MCK(cudaEventSynchronize(m->graphs_done));
    MCK(cudaStreamSynchronize(m->stream));
    MCK(cudaMemcpy(m->master, host, (size_t)MLP_NPARAM * 4, cudaMemcpyHostToDevice));
    int rc = refresh(m, m->stream);
    if (rc) return rc;
    MCK(cudaStreamSynchronize(m->stream));
    return SMC_OK;
}

int smc_mlp_gradient(smc_mlp *m, const float *x, const float *y, int n, float *grad_host, float *loss_host)
{
    if (!m || !x || !y || !grad_host || n < 1 || n > kMaxBatch) return SMC_E_INVALID_ARG;
    int rc = check_waits(m);
    if (rc) return rc;
    MCK(cudaSetDevice(m->device));
    if (m->graphs_done) MCK(cudaEventSynchronize(m->graphs_done));
    cudaStream_t s = m->stream;
    float *acc = m->loss + kMaxEpochs;
    MCK(cudaMemsetAsync(acc, 0, 4, s));
    StepRows rs{x, y, (uint64_t)n, m->n_in, n, 0, 0, 0, nullptr};
    int parts = 0;
    rc = step_launch(m, rs, acc, false, s, &parts);
    if (rc) return rc;
    mlp_update_kernel<<<kUpdBlocks, kUpdThreads, 0, s>>>(parts, m->part, m->master, m->am, m->av, 0.0f, 0.f,
                                                              0.f, 0.f, m->ctr, m->grad, m->w1b, m->w2b, m->w3b);
    MCK(cudaGetLastError());
    MCK(cudaMemcpyAsync(grad_host, m->grad, (size_t)MLP_NPARAM * 4, cudaMemcpyDeviceToHost, s));
    if (loss_host) MCK(cudaMemcpyAsync(loss_host, acc, 4, cudaMemcpyDeviceToHost, s));
    MCK(cudaStreamSynchronize(s));
    if (loss_host) *loss_host /= (float)n;
    return check_waits(m);
}

int smc_mlp_train(smc_mlp *m, const float *x, const float *y, uint64_t n, int epochs, int batch, float lr,
                  uint64_t seed, float *loss_host, void *stream)
{
    if (!m || !x || !y || n < 1 || epochs < 1 || epochs > kMaxEpochs || batch < 1 || batch > kMaxBatch ||
        !(lr > 0.0f))
        return SMC_E_INVALID_ARG;
    int rc = check_waits(m);
    if (rc) return rc;
    MCK(cudaSetDevice(m->device));
    cudaStream_t s = stream ? (cudaStream_t)stream : m->stream;
    const uint64_t steps = (n + batch - 1) / (uint64_t)batch;
    const int n_full = (int)std::min<uint64_t>(steps, kGraphSteps);
    const int n_rest = (int)(steps % (uint64_t)n_full);
    const StepRows rs{x, y, n, m->n_in, batch, 0, 1, seed, m->ctr};
    TrainGraphs &g = m->graphs;
    if (!(g.full && g.x == x && g.y == y && g.n == n && g.seed == seed && g.batch == batch && g.lr == lr &&
          g.n_full == n_full && g.n_rest == n_rest)) {
        drop_graphs(m);
        rc = capture_steps(m, rs, lr, n_full, &g.full);
        if (!rc) rc = capture_steps(m, rs, lr, n_rest, &g.rest);
        if (rc) {
            drop_graphs(m);
            return rc;
        }
        g.x = x, g.y = y, g.n = n, g.seed = seed, g.batch = batch, g.lr = lr, g.n_full = n_full, g.n_rest = n_rest;
    }
    // sampling step 0 (Adam's t carries over); the minibatch of step k of
    // the call is drawn from (seed, k)
    MCK(cudaMemsetAsync(m->ctr, 0, sizeof(unsigned long long), s));
    for (int ep = 0; ep < epochs; ++ep) {
        MCK(cudaMemsetAsync(m->loss + kMaxEpochs, 0, 4, s));
        for (uint64_t k = 0; k < steps / (uint64_t)n_full; ++k) MCK(cudaGraphLaunch(g.full, s));
        if (g.rest) MCK(cudaGraphLaunch(g.rest, s));
        MCK(cudaMemcpyAsync(m->loss + ep, m->loss + kMaxEpochs, 4, cudaMemcpyDeviceToDevice, s));
    }
    MCK(cudaEventRecord(m->graphs_done, s));
    if (loss_host) {
        MCK(cudaMemcpyAsync(loss_host, m->loss, (size_t)epochs * 4, cudaMemcpyDeviceToHost, s));
        MCK(cudaStreamSynchronize(s));
        for (int ep = 0; ep < epochs; ++ep) loss_host[ep] /= (float)(steps * (uint64_t)batch);
        return check_waits(m);
    }
    return SMC_OK;
}

int smc_mlp_predict_masked(smc_mlp *m, const float *x, uint64_t n, const uint8_t *skip, float *g, void *stream)
{
    if (!m || (n && (!x || !g))) return SMC_E_INVALID_ARG;
    int rc = check_waits(m);
    if (rc) return rc;
    if (n == 0) return SMC_OK;
    MCK(cudaSetDevice(m->device));
    cudaStream_t s = stream ? (cudaStream_t)stream : m->stream;
    // one CTA per SM (its shared memory rules out a second, which its
    // allocation of the whole tensor memory requires)
    const uint64_t tiles = (n + kTcRows - 1) / kTcRows;
    const uint64_t want = (tiles + kTcGroups - 1) / kTcGroups;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)m->n_sm));
    mlp_tc_forward<<<grid, kTcThreads, kTcSmem, s>>>(x, n, m->n_in, skip, m->w1b, m->w2b, m->w3b, m->master, g,
                                                     m->d_err);
    MCK(cudaGetLastError());
    return SMC_OK;
}

int smc_mlp_predict(smc_mlp *m, const float *x, uint64_t n, float *g, void *stream)
{
    return smc_mlp_predict_masked(m, x, n, nullptr, g, stream);
}

}  // extern "C"
