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
constexpr int kTcSmBar = kTcSmB4 + 16 * 16 * 2;        // one mbarrier per pipeline, then the TMEM address
constexpr int kTcSmGroup = (kTcSmBar + 8 * kTcGroups + 4 + 1023) / 1024 * 1024;
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

// stages an N x K row-major BF16 matrix (global) into the core-matrix layout
__device__ __forceinline__ void tc_stage_operand(unsigned char *dst, const bf16 *src, int N, int K)
{
    const int chunks = N * (K / 8);
    for (int i = threadIdx.x; i < chunks; i += blockDim.x) {
        const int r = i / (K / 8), kg = i % (K / 8);
        *reinterpret_cast<uint4 *>(dst + tc_core_offset(r, kg, K)) =
            *reinterpret_cast<const uint4 *>(src + (size_t)r * K + kg * 8);
    }
}

// element (r, k) of an operand with K columns in the core-matrix layout
__device__ __forceinline__ bf16 *tc_elem(unsigned char *base, int r, int k, int K)
{
    return reinterpret_cast<bf16 *>(base + tc_elem_offset(r, k, K));
}

// high and low BF16 parts of an FP32 value (v = hi + lo to about 2^-17 relative)
__device__ __forceinline__ bf16 bf16_hi(float v) { return __float2bfloat16_rn(v); }
__device__ __forceinline__ bf16 bf16_lo(float v) { return __float2bfloat16_rn(v - __bfloat162float(__float2bfloat16_rn(v))); }

// The training pass's tiles in global memory: per 128-row tile t, the input
// (4 KB at x + t * 4096) and each layer's activations and deltas (32 KB at
// h1 + t * 32768, ...), every one in the K-major core-matrix layout of
// smc_tc.h with the rows as M, so that the backward and weight-gradient
// kernels read them into shared memory unchanged; the logits z and the
// output deltas dz per row.
struct TrainTiles {
    unsigned char *x, *h1, *h2, *h3, *d1, *d2, *d3;
    float *z, *dz;
};
constexpr int kTileX = kTcRows * IN * 2, kTileH = kTcRows * H * 2;

// The forward pass over n rows, one persistent launch (one CTA of
// kTcThreads per SM) over 128-row tiles, weights staged once per CTA.
// Inference (TRAIN = false): FP32 features x [n][n_in] (n_in <= 16), rounded
// to BF16 as the training input is; g[r] = 1 / (1 + e^-z); rows with
// skip[r] != 0 (skip may be null) need no output, and a tile whose rows all
// skip is not computed.  Training (TRAIN = true): BF16 rows xb [n][16]; the
// input and activation tiles and the logits go to tt.  A wait that gives up
// sets *err and leaves NaN in the outputs of the tile it was working on,
// and that pipeline stops.
template <bool TRAIN>
__global__ void __launch_bounds__(kTcThreads) mlp_tc_forward(const float *__restrict__ x,
                                                             const bf16 *__restrict__ xb, uint64_t n, int n_in,
                                                             const uint8_t *__restrict__ skip, const bf16 *w1b,
                                                             const bf16 *w2b, const bf16 *w3b, const float *master,
                                                             float *g_out, TrainTiles tt, int *err)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + kTcSmBar);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + kTcSmBar + 8 * kTcGroups);
    const int tid = threadIdx.x, warp = tid >> 5, grp = tid >> 7, gt = tid & 127;
    const int bid = 1 + grp;  // the pipeline's named barrier

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < kTcGroups; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bars + i)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_stage_operand(sm + kTcSmW1, w1b, H, IN);
    tc_stage_operand(sm + kTcSmW2, w2b, H, H);
    tc_stage_operand(sm + kTcSmW3, w3b, H, H);
    const bf16 zero = __float2bfloat16_rn(0.0f), one = __float2bfloat16_rn(1.0f);
    for (int i = tid; i < H * 16; i += blockDim.x) {  // ones, bias tiles (rows x 16 columns)
        const int r = i >> 4, k = i & 15;
        *tc_elem(sm + kTcSmOnes, r, k, 16) = k < 2 ? one : zero;
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            const float b = master[MLP_OFF_B1 + l * (H * H + H) + r];
            *tc_elem(sm + kTcSmB1 + l * H * 16 * 2, r, k, 16) = k == 0 ? bf16_hi(b) : k == 1 ? bf16_lo(b) : zero;
        }
    }
    for (int i = tid; i < 16 * H; i += blockDim.x) {  // output unit: rows 0, 1 = w4 high, low
        const int r = i / H, k = i % H;
        const float w = master[MLP_OFF_W4 + k];
        *tc_elem(sm + kTcSmW4, r, k, H) = r == 0 ? bf16_hi(w) : r == 1 ? bf16_lo(w) : zero;
    }
    for (int i = tid; i < 16 * 16; i += blockDim.x) {
        const int r = i >> 4, k = i & 15;
        const float b = master[MLP_OFF_B4];
        *tc_elem(sm + kTcSmB4, r, k, 16) = (r == 0 && k == 0) ? bf16_hi(b) : (r == 0 && k == 1) ? bf16_lo(b) : zero;
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t tacc = tmem + 128u * grp;                              // the pipeline's columns
    const uint32_t t_row = tacc + ((uint32_t)(32 * (warp & 3)) << 16);  // this warp's 32 lanes

    unsigned char *act = sm + kTcSmGroup + grp * kTcGroupBytes;
    const uint32_t bar = smem_u32(bars + grp);
    const uint32_t aAct = smem_u32(act), aOnes = smem_u32(sm + kTcSmOnes);
    uint32_t phase = 0;
    bool failed = false;
    const uint64_t tiles = (n + kTcRows - 1) / kTcRows;

    // a tile's features and mask are loaded one tile ahead, so their
    // latency overlaps the previous tile's layers
    const uint64_t stride = (uint64_t)gridDim.x * kTcGroups;
    auto load_tile = [&](uint64_t t, float (&f)[IN], bool &nd) {
        const uint64_t r = t * kTcRows + gt;
        if constexpr (TRAIN) {
            nd = r < n;
            const uint4 *src = reinterpret_cast<const uint4 *>(xb + r * IN);
            const uint4 v0 = nd ? src[0] : make_uint4(0, 0, 0, 0), v1 = nd ? src[1] : make_uint4(0, 0, 0, 0);
            const uint32_t w[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
            for (int k = 0; k < IN / 2; ++k) {  // exact: the values are BF16 already
                const float2 p = unpack2(w[k]);
                f[2 * k] = p.x;
                f[2 * k + 1] = p.y;
            }
        } else {
            nd = r < n && !(skip && skip[r]);
#pragma unroll
            for (int k = 0; k < IN; ++k) f[k] = (r < n && k < n_in) ? x[r * n_in + k] : 0.0f;
        }
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
                if constexpr (TRAIN)
                    *reinterpret_cast<uint4 *>(tt.x + tile * kTileX + tc_core_offset(gt, kg, IN)) = v;
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
                unsigned char *hg = nullptr;  // training: this layer's tile in global memory
                if constexpr (TRAIN) hg = (layer == 0 ? tt.h1 : layer == 1 ? tt.h2 : tt.h3) + tile * kTileH;
                auto store_chunk = [&](int c, const uint32_t (&v)[32]) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const uint4 w =
                            make_uint4(relu_pack2(v[8 * q], v[8 * q + 1]), relu_pack2(v[8 * q + 2], v[8 * q + 3]),
                                       relu_pack2(v[8 * q + 4], v[8 * q + 5]), relu_pack2(v[8 * q + 6], v[8 * q + 7]));
                        *reinterpret_cast<uint4 *>(act + tc_core_offset(gt, 4 * c + q, H)) = w;
                        if constexpr (TRAIN) *reinterpret_cast<uint4 *>(hg + tc_core_offset(gt, 4 * c + q, H)) = w;
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
            if (row < n) (TRAIN ? tt.z : g_out)[row] = __int_as_float(0x7fc00000);
            if (gt == 0) atomicExch(err, 1);
            break;
        }
        const float z = __uint_as_float(zc[0]) + __uint_as_float(zc[1]);
        if constexpr (TRAIN) {
            if (need) tt.z[row] = z;
        } else {
            if (need) g_out[row] = 1.0f / (1.0f + expf(-z));
        }
    }
    // Release tensor memory once every MMA and load of this CTA has finished.
    // A pipeline that gave up waits again (bounded) for the completion of its
    // last committed MMAs: up to four more periods of kTcWaitNs.  Only if the
    // tensor cores never report it does the CTA release the memory without
    // the confirmation (a CTA may not exit holding tensor memory), and it
    // records that case (err = 2) for the host.
    if (failed && gt == 0) {
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

// Sums the partial gradients (one per weight-gradient CTA), optionally
// applies Adam (lr > 0) to the FP32 master weights, and refreshes their BF16
// copies (row-major; the kernels stage them in the operand layout and read
// them MN-major where they need the transpose).
__global__ void mlp_update_kernel(int nparts, const float *part, float *master, float *am, float *av, float lr,
                                  float beta1, float beta2, float eps, float bc1, float bc2, float *grad_out,
                                  bf16 *w1b, bf16 *w2b, bf16 *w3b)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= MLP_NPARAM) return;
    float gsum = 0.0f;
    for (int c = 0; c < nparts; ++c) gsum += part[(size_t)c * MLP_NPARAM + i];
    if (grad_out) grad_out[i] = gsum;
    float w = master[i];
    if (lr > 0.0f) {
        const float m = beta1 * am[i] + (1.0f - beta1) * gsum;
        const float v = beta2 * av[i] + (1.0f - beta2) * gsum * gsum;
        am[i] = m;
        av[i] = v;
        w -= lr * (m / bc1) / (sqrtf(v / bc2) + eps);
        master[i] = w;
    }
    const bf16 wb = __float2bfloat16(w);
    if (i < MLP_OFF_B1) w1b[i - MLP_OFF_W1] = wb;
    else if (i >= MLP_OFF_W2 && i < MLP_OFF_B2) w2b[i - MLP_OFF_W2] = wb;
    else if (i >= MLP_OFF_W3 && i < MLP_OFF_B3) w3b[i - MLP_OFF_W3] = wb;
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Rows of x (FP32 [n][n_in]) into the BF16 input buffer [B][16] (zero
// padded): row i of the batch is row i + base (predict), or a row drawn with
// replacement from a counter-based hash of (seed, step, i) (training).
__global__ void mlp_gather_kernel(const float *x, const float *y, uint64_t n, int n_in, int B, uint64_t base,
                                  int sample, uint64_t seed, uint64_t step, bf16 *xb, float *yb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B) return;
    uint64_t r;
    if (sample) r = splitmix64(seed ^ splitmix64(step * 0x100000001ull + (uint64_t)i)) % n;
    else r = base + (uint64_t)i;
    const bool ok = r < n;
#pragma unroll
    for (int k = 0; k < IN; ++k) xb[(size_t)i * IN + k] = __float2bfloat16(ok && k < n_in ? x[r * n_in + k] : 0.0f);
    if (yb) yb[i] = ok ? y[r] : 0.0f;
}

constexpr int kMaxBatch = 65536;                             // rows per training step
constexpr int kMaxTiles = kMaxBatch / kTcRows;
constexpr int kMaxParts = 256;                               // weight-gradient CTAs (one per SM)

}  // namespace

struct smc_mlp {
    int device = 0;
    int n_in = 0;
    int n_sm = 0;
    std::string err;
    cudaStream_t stream = nullptr;
    float *master = nullptr, *am = nullptr, *av = nullptr, *part = nullptr, *grad = nullptr;
    bf16 *w1b = nullptr, *w2b = nullptr, *w3b = nullptr;
    bf16 *xb = nullptr;    // the minibatch's rows, BF16 [kMaxBatch][16]
    float *yb = nullptr, *loss = nullptr;
    TrainTiles tt{};       // saved tiles of the training step (kMaxTiles each)
    int *h_err = nullptr, *d_err = nullptr;  // a tensor-core wait gave up (mapped host memory)
    uint64_t adam_t = 0;
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
    mlp_update_kernel<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(0, m->part, m->master, m->am, m->av, 0.0f, 0.f,
                                                              0.f, 0.f, 1.f, 1.f, nullptr, m->w1b, m->w2b, m->w3b);
    MCK(cudaGetLastError());
    return SMC_OK;
}

// One forward, backward and weight-gradient pass over the B rows already
// gathered into xb / yb (the loss sum added to *loss_acc); *nparts = the
// partial gradients written to part.
int train_pass(smc_mlp *m, int B, float *loss_acc, cudaStream_t s, int *nparts)
{
    const int tiles = (B + kTcRows - 1) / kTcRows;
    const int grid_rows = std::max(1, std::min((tiles + kTcGroups - 1) / kTcGroups, m->n_sm));
    mlp_tc_forward<true><<<grid_rows, kTcThreads, kTcSmem, s>>>(nullptr, m->xb, (uint64_t)B, IN, nullptr, m->w1b,
                                                               m->w2b, m->w3b, m->master, nullptr, m->tt, m->d_err);
    MCK(cudaGetLastError());
    mlp_train_bwd_kernel<<<grid_rows, kTcThreads, kBwSmem, s>>>(m->yb, (uint64_t)B, 1.0f / (float)B, m->w2b, m->w3b,
                                                               m->master, m->tt, loss_acc, m->d_err);
    MCK(cudaGetLastError());
    const int parts = std::max(1, std::min(tiles, std::min(m->n_sm, kMaxParts)));
    mlp_train_wgrad_kernel<<<parts, 128, kWgSmem, s>>>((uint64_t)tiles, m->tt, m->part, m->d_err);
    MCK(cudaGetLastError());
    *nparts = parts;
    return SMC_OK;
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
    const size_t np = MLP_NPARAM;
    void **f32[] = {(void **)&m->master, (void **)&m->am, (void **)&m->av, (void **)&m->grad};
    for (void **p : f32)
        if (cudaMalloc(p, np * 4) != cudaSuccess) return fin(SMC_E_OOM);
    if (cudaMalloc((void **)&m->part, (size_t)kMaxParts * np * 4) != cudaSuccess) return fin(SMC_E_OOM);
    void **wb[] = {(void **)&m->w1b, (void **)&m->w2b, (void **)&m->w3b};
    for (void **p : wb)
        if (cudaMalloc(p, (size_t)H * H * 2) != cudaSuccess) return fin(SMC_E_OOM);
    if (cudaMalloc((void **)&m->xb, (size_t)kMaxBatch * IN * 2) != cudaSuccess) return fin(SMC_E_OOM);
    if (cudaMalloc((void **)&m->yb, (size_t)kMaxBatch * 4) != cudaSuccess) return fin(SMC_E_OOM);
    if (cudaMalloc((void **)&m->tt.x, (size_t)kMaxTiles * kTileX) != cudaSuccess) return fin(SMC_E_OOM);
    unsigned char **tiles[] = {&m->tt.h1, &m->tt.h2, &m->tt.h3, &m->tt.d1, &m->tt.d2, &m->tt.d3};
    for (unsigned char **p : tiles)
        if (cudaMalloc((void **)p, (size_t)kMaxTiles * kTileH) != cudaSuccess) return fin(SMC_E_OOM);
    if (cudaMalloc((void **)&m->tt.z, (size_t)kMaxBatch * 4) != cudaSuccess) return fin(SMC_E_OOM);
    if (cudaMalloc((void **)&m->tt.dz, (size_t)kMaxBatch * 4) != cudaSuccess) return fin(SMC_E_OOM);
    if (cudaMalloc((void **)&m->loss, 4096 * 4) != cudaSuccess) return fin(SMC_E_OOM);
    if (cudaHostAlloc((void **)&m->h_err, sizeof(int), cudaHostAllocMapped) != cudaSuccess) return fin(SMC_E_OOM);
    *m->h_err = 0;
    if (cudaHostGetDevicePointer((void **)&m->d_err, m->h_err, 0) != cudaSuccess) return fin(SMC_E_CUDA);
    if (cudaDeviceGetAttribute(&m->n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return fin(SMC_E_CUDA);
    const void *kern[] = {(const void *)mlp_tc_forward<false>, (const void *)mlp_tc_forward<true>,
                          (const void *)mlp_train_bwd_kernel, (const void *)mlp_train_wgrad_kernel};
    const int smem[] = {kTcSmem, kTcSmem, kBwSmem, kWgSmem};
    for (int k = 0; k < 4; ++k)
        if (cudaFuncSetAttribute(kern[k], cudaFuncAttributeMaxDynamicSharedMemorySize, smem[k]) != cudaSuccess)
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
    void *ptrs[] = {m->master, m->am, m->av, m->part, m->grad, m->w1b, m->w2b, m->w3b, m->xb, m->yb, m->loss,
                    m->tt.x, m->tt.h1, m->tt.h2, m->tt.h3, m->tt.d1, m->tt.d2, m->tt.d3, m->tt.z, m->tt.dz};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (m->h_err) cudaFreeHost(m->h_err);
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
    MCK(cudaStreamSynchronize(m->stream));
    MCK(cudaMemcpy(host, m->master, (size_t)MLP_NPARAM * 4, cudaMemcpyDeviceToHost));
    return SMC_OK;
}

int smc_mlp_set_params(smc_mlp *m, const float *host)
{
    if (!m || !host) return SMC_E_INVALID_ARG;
    MCK(cudaSetDevice(m->device));
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
    cudaStream_t s = m->stream;
    mlp_gather_kernel<<<(n + 127) / 128, 128, 0, s>>>(x, y, (uint64_t)n, m->n_in, n, 0, 0, 0, 0, m->xb, m->yb);
    MCK(cudaGetLastError());
    MCK(cudaMemsetAsync(m->loss, 0, 4, s));
    int parts = 0;
    rc = train_pass(m, n, m->loss, s, &parts);
    if (rc) return rc;
    mlp_update_kernel<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(parts, m->part, m->master, m->am, m->av, 0.0f, 0.f,
                                                              0.f, 0.f, 1.f, 1.f, m->grad, m->w1b, m->w2b, m->w3b);
    MCK(cudaGetLastError());
    MCK(cudaMemcpyAsync(grad_host, m->grad, (size_t)MLP_NPARAM * 4, cudaMemcpyDeviceToHost, s));
    if (loss_host) MCK(cudaMemcpyAsync(loss_host, m->loss, 4, cudaMemcpyDeviceToHost, s));
    MCK(cudaStreamSynchronize(s));
    if (loss_host) *loss_host /= (float)n;
    return check_waits(m);
}

int smc_mlp_train(smc_mlp *m, const float *x, const float *y, uint64_t n, int epochs, int batch, float lr,
                  uint64_t seed, float *loss_host, void *stream)
{
    if (!m || !x || !y || n < 1 || epochs < 1 || epochs > 4096 || batch < 1 || batch > kMaxBatch || !(lr > 0.0f))
        return SMC_E_INVALID_ARG;
    int rc = check_waits(m);
    if (rc) return rc;
    MCK(cudaSetDevice(m->device));
    cudaStream_t s = stream ? (cudaStream_t)stream : m->stream;
    const uint64_t steps = (n + batch - 1) / (uint64_t)batch;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    MCK(cudaMemsetAsync(m->loss, 0, (size_t)epochs * 4, s));
    for (int ep = 0; ep < epochs; ++ep) {
        for (uint64_t st = 0; st < steps; ++st) {
            const uint64_t step_id = (uint64_t)ep * steps + st;
            mlp_gather_kernel<<<(batch + 127) / 128, 128, 0, s>>>(x, y, n, m->n_in, batch, 0, 1, seed, step_id,
                                                                  m->xb, m->yb);
            MCK(cudaGetLastError());
            int parts = 0;
            rc = train_pass(m, batch, m->loss + ep, s, &parts);
            if (rc) return rc;
            ++m->adam_t;
            const float bc1 = 1.0f - std::pow(b1, (float)m->adam_t), bc2 = 1.0f - std::pow(b2, (float)m->adam_t);
            mlp_update_kernel<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(parts, m->part, m->master, m->am, m->av, lr,
                                                                      b1, b2, eps, bc1, bc2, nullptr, m->w1b,
                                                                      m->w2b, m->w3b);
            MCK(cudaGetLastError());
        }
    }
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
    mlp_tc_forward<false><<<grid, kTcThreads, kTcSmem, s>>>(x, nullptr, n, m->n_in, skip, m->w1b, m->w2b, m->w3b,
                                                            m->master, g, TrainTiles{}, m->d_err);
    MCK(cudaGetLastError());
    return SMC_OK;
}

int smc_mlp_predict(smc_mlp *m, const float *x, uint64_t n, float *g, void *stream)
{
    return smc_mlp_predict_masked(m, x, n, nullptr, g, stream);
}

}  // extern "C"
