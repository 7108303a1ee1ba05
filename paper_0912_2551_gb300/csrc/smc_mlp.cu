// smc_mlp.cu -- the surrogate network used as a control variate: forward,
// backward and Adam update as hand-written BF16 tensor-core kernels with
// FP32 accumulation and FP32 master weights.  Inference (on the estimator's
// path) runs on tcgen05 with the accumulator in tensor memory; training
// (tiny minibatches) runs on mma.sync m16n8k16.
//
// Network: g(x) = sigmoid(w4 . h3 + b4), h_l = relu(W_l h_{l-1} + b_l),
// x in R^16 (zero-padded features), hidden width 128.  Training minimises the
// binary cross-entropy of g against the trajectory verdicts.
//
// Fragment layout of mma.m16n8k16 (g = lane / 4, t = lane % 4):
//   A 16x16 row-major: a0 (g, 2t..2t+1), a1 (g+8, 2t..), a2 (g, 2t+8..), a3 (g+8, 2t+8..)
//   B 16x8  col-major: b0 (k = 2t..2t+1, n = g), b1 (k = 2t+8.., n = g)
//   C 16x8:            c0 (g, 2t), c1 (g, 2t+1), c2 (g+8, 2t), c3 (g+8, 2t+1)
// so two adjacent C tiles of one layer are exactly one A k-tile of the next:
// activations go from accumulator to operand registers without shared memory.
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

constexpr int H = MLP_H, IN = MLP_IN, LDC = MLP_CHUNK + 8;

__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ float2 unpack2(uint32_t w)
{
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w));
}

__device__ __forceinline__ uint32_t ld32(const bf16 *p) { return *reinterpret_cast<const uint32_t *>(p); }
__device__ __forceinline__ void st32(bf16 *p, uint32_t v) { *reinterpret_cast<uint32_t *>(p) = v; }

// copies n bytes (multiple of 16) global -> shared
__device__ __forceinline__ void stage(void *dst, const void *src, int n)
{
    const uint4 *s = reinterpret_cast<const uint4 *>(src);
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    for (int i = threadIdx.x; i < n / 16; i += blockDim.x) d[i] = s[i];
}

// bias + relu on a 16 x 128 accumulator slab, BF16 rounding, optional store
// of the activations, and repacking as the next layer's A fragments.
__device__ __forceinline__ void relu_epilogue(float (&acc)[16][4], const float *bias, bf16 *hout, int ra,
                                              int rb, int B, int t, uint32_t (&af)[8][4])
{
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
        const int col = 8 * nt + 2 * t;
        const float v0 = fmaxf(acc[nt][0] + bias[col], 0.0f), v1 = fmaxf(acc[nt][1] + bias[col + 1], 0.0f);
        const float v2 = fmaxf(acc[nt][2] + bias[col], 0.0f), v3 = fmaxf(acc[nt][3] + bias[col + 1], 0.0f);
        const uint32_t pa = pack2(v0, v1), pb = pack2(v2, v3);
        if (hout) {
            if (ra < B) st32(hout + (size_t)ra * H + col, pa);
            if (rb < B) st32(hout + (size_t)rb * H + col, pb);
        }
        if ((nt & 1) == 0) { af[nt >> 1][0] = pa; af[nt >> 1][1] = pb; }
        else { af[nt >> 1][2] = pa; af[nt >> 1][3] = pb; }
    }
}

// Weights of the network staged in shared memory (forward direction):
// W1 [H][IN], W2 [H][H], W3 [H][H] in BF16, then b1 | b2 | b3 | w4 | b4 in FP32.
__device__ __forceinline__ void stage_forward_weights(unsigned char *sm, const bf16 *w1b, const bf16 *w2b,
                                                      const bf16 *w3b, const float *master)
{
    bf16 *sW1 = reinterpret_cast<bf16 *>(sm);
    bf16 *sW2 = sW1 + H * IN;
    bf16 *sW3 = sW2 + H * H;
    float *sb = reinterpret_cast<float *>(sW3 + H * H);
    stage(sW1, w1b, H * IN * 2);
    stage(sW2, w2b, H * H * 2);
    stage(sW3, w3b, H * H * 2);
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        sb[i] = master[MLP_OFF_B1 + i];
        sb[H + i] = master[MLP_OFF_B2 + i];
        sb[2 * H + i] = master[MLP_OFF_B3 + i];
        sb[3 * H + i] = master[MLP_OFF_W4 + i];
    }
    if (threadIdx.x == 0) sb[4 * H] = master[MLP_OFF_B4];
    __syncthreads();
}

// The network on one 16-row tile held by a warp: a = the input A fragment of
// rows ra = r0 + g and rb = r0 + g + 8.  The logits of rows ra / rb end up in
// za / zb (every lane of the row's quad).  Stores h1..h3 (rows < B) when the
// pointers are given.
__device__ __forceinline__ void forward_tile(const uint32_t (&a)[4], const unsigned char *sm, int g, int t, int ra,
                                             int rb, int B, bf16 *h1, bf16 *h2, bf16 *h3, float &za_out,
                                             float &zb_out)
{
    const bf16 *sW1 = reinterpret_cast<const bf16 *>(sm);
    const bf16 *sW2 = sW1 + H * IN;
    const bf16 *sW3 = sW2 + H * H;
    const float *sb = reinterpret_cast<const float *>(sW3 + H * H);
    float acc[16][4];
    uint32_t af[8][4];
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
        acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
        const bf16 *w = sW1 + (8 * nt + g) * IN + 2 * t;
        mma16816(acc[nt], a, ld32(w), ld32(w + 8));
    }
    relu_epilogue(acc, sb, h1, ra, rb, B, t, af);
#pragma unroll 1
    for (int layer = 0; layer < 2; ++layer) {
        const bf16 *sW = layer == 0 ? sW2 : sW3;
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
#pragma unroll
        for (int kt = 0; kt < 8; ++kt)
#pragma unroll
            for (int nt = 0; nt < 16; ++nt) {
                const bf16 *w = sW + (8 * nt + g) * H + 16 * kt + 2 * t;
                mma16816(acc[nt], af[kt], ld32(w), ld32(w + 8));
            }
        relu_epilogue(acc, sb + (layer + 1) * H, layer == 0 ? h2 : h3, ra, rb, B, t, af);
    }
    // output unit from the BF16 activations of the last hidden layer
    float za = 0.0f, zb = 0.0f;
#pragma unroll
    for (int kt = 0; kt < 8; ++kt) {
        const int c0 = 16 * kt + 2 * t, c1 = c0 + 8;
        const float2 p0 = unpack2(af[kt][0]), p1 = unpack2(af[kt][1]);
        const float2 p2 = unpack2(af[kt][2]), p3 = unpack2(af[kt][3]);
        const float *w4 = sb + 3 * H;
        za += p0.x * w4[c0] + p0.y * w4[c0 + 1] + p2.x * w4[c1] + p2.y * w4[c1 + 1];
        zb += p1.x * w4[c0] + p1.y * w4[c0 + 1] + p3.x * w4[c1] + p3.y * w4[c1 + 1];
    }
    za += __shfl_xor_sync(0xffffffffu, za, 1);
    za += __shfl_xor_sync(0xffffffffu, za, 2);
    zb += __shfl_xor_sync(0xffffffffu, zb, 1);
    zb += __shfl_xor_sync(0xffffffffu, zb, 2);
    za_out = za + sb[4 * H];
    zb_out = zb + sb[4 * H];
}

// Forward pass over B rows of x (BF16 [B][16]).  z_out[r] = logit.  With
// train, the activations h1..h3 are stored for the backward pass.
__global__ void __launch_bounds__(128) mlp_fwd_kernel(const bf16 *__restrict__ x, int B, const bf16 *w1b,
                                                      const bf16 *w2b, const bf16 *w3b, const float *master,
                                                      float *z_out, bf16 *h1, bf16 *h2, bf16 *h3)
{
    extern __shared__ __align__(16) unsigned char sm[];
    stage_forward_weights(sm, w1b, w2b, w3b, master);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int r0 = blockIdx.x * MLP_ROWS_FWD + warp * 16, ra = r0 + g, rb = r0 + g + 8;
    if (r0 >= B) return;
    uint32_t a[4];
    a[0] = ra < B ? ld32(x + (size_t)ra * IN + 2 * t) : 0u;
    a[1] = rb < B ? ld32(x + (size_t)rb * IN + 2 * t) : 0u;
    a[2] = ra < B ? ld32(x + (size_t)ra * IN + 2 * t + 8) : 0u;
    a[3] = rb < B ? ld32(x + (size_t)rb * IN + 2 * t + 8) : 0u;
    float za, zb;
    forward_tile(a, sm, g, t, ra, rb, B, h1, h2, h3, za, zb);
    if (t == 0) {
        if (ra < B) z_out[ra] = za;
        if (rb < B) z_out[rb] = zb;
    }
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

// Inference over n rows of FP32 features x [n][n_in] (n_in <= 16): one
// persistent launch (one CTA of kTcThreads per SM) over 128-row tiles,
// weights staged once per CTA, features rounded to BF16 as the training
// input is; g[r] = 1 / (1 + e^-z).  Rows with skip[r] != 0 (may be null)
// need no output; a tile whose rows all skip is not computed.  A wait that
// gives up sets *err and leaves NaN in the outputs of the tile it was
// working on, and that pipeline stops.
__global__ void __launch_bounds__(kTcThreads) mlp_infer_kernel(const float *__restrict__ x, uint64_t n, int n_in,
                                                               const uint8_t *__restrict__ skip, const bf16 *w1b,
                                                               const bf16 *w2b, const bf16 *w3b,
                                                               const float *master, float *g_out, int *err)
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
                    for (int q = 0; q < 4; ++q)
                        *reinterpret_cast<uint4 *>(act + tc_core_offset(gt, 4 * c + q, H)) =
                            make_uint4(relu_pack2(v[8 * q], v[8 * q + 1]), relu_pack2(v[8 * q + 2], v[8 * q + 3]),
                                       relu_pack2(v[8 * q + 4], v[8 * q + 5]), relu_pack2(v[8 * q + 6], v[8 * q + 7]));
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

// Backward pass for the activations: dz = (sigmoid(z) - y) / B (the mean
// binary cross-entropy), dh3 = dz w4 . [h3 > 0], dh2 = (dh3 W3) . [h2 > 0],
// dh1 = (dh2 W2) . [h1 > 0]; stored in BF16 for the weight gradients.
// loss_acc accumulates the summed cross-entropy.
__global__ void __launch_bounds__(128) mlp_bwd_kernel(const float *z, const float *y, int B, float inv_b,
                                                      const bf16 *h1, const bf16 *h2, const bf16 *h3,
                                                      const bf16 *w2t, const bf16 *w3t, const float *master,
                                                      float *dz_out, bf16 *dh1, bf16 *dh2, bf16 *dh3,
                                                      float *loss_acc)
{
    extern __shared__ __align__(16) unsigned char sm[];
    bf16 *sW3T = reinterpret_cast<bf16 *>(sm);
    bf16 *sW2T = sW3T + H * H;
    float *sw4 = reinterpret_cast<float *>(sW2T + H * H);
    stage(sW3T, w3t, H * H * 2);
    stage(sW2T, w2t, H * H * 2);
    for (int i = threadIdx.x; i < H; i += blockDim.x) sw4[i] = master[MLP_OFF_W4 + i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int r0 = blockIdx.x * MLP_ROWS_FWD + warp * 16, ra = r0 + g, rb = r0 + g + 8;
    if (r0 >= B) return;

    float dza = 0.0f, dzb = 0.0f, loss = 0.0f;
    if (ra < B) {
        const float zz = z[ra], yy = y[ra];
        dza = (1.0f / (1.0f + expf(-zz)) - yy) * inv_b;
        loss += fmaxf(zz, 0.0f) - zz * yy + log1pf(expf(-fabsf(zz)));
    }
    if (rb < B) {
        const float zz = z[rb], yy = y[rb];
        dzb = (1.0f / (1.0f + expf(-zz)) - yy) * inv_b;
        loss += fmaxf(zz, 0.0f) - zz * yy + log1pf(expf(-fabsf(zz)));
    }
    if (t == 0) {
        if (ra < B) dz_out[ra] = dza;
        if (rb < B) dz_out[rb] = dzb;
        if (loss != 0.0f) atomicAdd(loss_acc, loss);
    }
    uint32_t ag[8][4];
#pragma unroll
    for (int kt = 0; kt < 8; ++kt)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int row = (q & 1) ? rb : ra;
            const int col = 16 * kt + 2 * t + ((q & 2) ? 8 : 0);
            const float d = (q & 1) ? dzb : dza;
            const float2 hv = unpack2(row < B ? ld32(h3 + (size_t)row * H + col) : 0u);
            const uint32_t pk = pack2(hv.x > 0.0f ? d * sw4[col] : 0.0f, hv.y > 0.0f ? d * sw4[col + 1] : 0.0f);
            ag[kt][q] = pk;
            if (row < B) st32(dh3 + (size_t)row * H + col, pk);
        }
    float acc[16][4];
#pragma unroll 1
    for (int layer = 0; layer < 2; ++layer) {
        const bf16 *sWT = layer == 0 ? sW3T : sW2T;
        const bf16 *hm = layer == 0 ? h2 : h1;
        bf16 *dout = layer == 0 ? dh2 : dh1;
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
#pragma unroll
        for (int kt = 0; kt < 8; ++kt)
#pragma unroll
            for (int nt = 0; nt < 16; ++nt) {
                const bf16 *w = sWT + (8 * nt + g) * H + 16 * kt + 2 * t;
                mma16816(acc[nt], ag[kt], ld32(w), ld32(w + 8));
            }
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) {
            const int col = 8 * nt + 2 * t;
            const float2 ma = unpack2(ra < B ? ld32(hm + (size_t)ra * H + col) : 0u);
            const float2 mb = unpack2(rb < B ? ld32(hm + (size_t)rb * H + col) : 0u);
            const uint32_t pa = pack2(ma.x > 0.0f ? acc[nt][0] : 0.0f, ma.y > 0.0f ? acc[nt][1] : 0.0f);
            const uint32_t pb = pack2(mb.x > 0.0f ? acc[nt][2] : 0.0f, mb.y > 0.0f ? acc[nt][3] : 0.0f);
            if (ra < B) st32(dout + (size_t)ra * H + col, pa);
            if (rb < B) st32(dout + (size_t)rb * H + col, pb);
            if ((nt & 1) == 0) { ag[nt >> 1][0] = pa; ag[nt >> 1][1] = pb; }
            else { ag[nt >> 1][2] = pa; ag[nt >> 1][3] = pb; }
        }
    }
}

// Weight gradients of layer L = blockIdx.y + 1 over a chunk of MLP_CHUNK rows:
// dW_L[o][i] = sum_r dh_L[r][o] h_{L-1}[r][i] (tensor cores, operands staged
// feature-major in shared memory), db_L[o] = sum_r dh_L[r][o]; layer 3 also
// dw4[i] = sum_r dz[r] h3[r][i] and db4 = sum_r dz[r].  Each chunk writes its
// own slice of part[chunk][param]; the Adam kernel sums the chunks.
__global__ void __launch_bounds__(256) mlp_wgrad_kernel(int B, const bf16 *x, const bf16 *h1, const bf16 *h2,
                                                        const bf16 *h3, const bf16 *dh1, const bf16 *dh2,
                                                        const bf16 *dh3, const float *dz, float *part)
{
    extern __shared__ __align__(16) unsigned char sm[];
    bf16 *sD = reinterpret_cast<bf16 *>(sm);  // [H][LDC]  dh, feature-major
    bf16 *sHp = sD + H * LDC;                 // [N][LDC]  h_{L-1}, feature-major
    const int L = blockIdx.y + 1, chunk = blockIdx.x, r0 = chunk * MLP_CHUNK;
    const bf16 *dh = L == 1 ? dh1 : (L == 2 ? dh2 : dh3);
    const bf16 *hp = L == 1 ? x : (L == 2 ? h1 : h2);
    const int N = L == 1 ? IN : H;
    const bf16 zero = __float2bfloat16(0.0f);
    for (int idx = threadIdx.x; idx < MLP_CHUNK * H; idx += blockDim.x) {
        const int r = idx / H, o = idx % H;
        sD[o * LDC + r] = (r0 + r < B) ? dh[(size_t)(r0 + r) * H + o] : zero;
    }
    for (int idx = threadIdx.x; idx < MLP_CHUNK * N; idx += blockDim.x) {
        const int r = idx / N, i = idx % N;
        sHp[i * LDC + r] = (r0 + r < B) ? hp[(size_t)(r0 + r) * N + i] : zero;
    }
    __syncthreads();
    float *out = part + (size_t)chunk * MLP_NPARAM;
    const int offW = L == 1 ? MLP_OFF_W1 : (L == 2 ? MLP_OFF_W2 : MLP_OFF_W3);
    const int offB = L == 1 ? MLP_OFF_B1 : (L == 2 ? MLP_OFF_B2 : MLP_OFF_B3);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int m0 = 16 * warp;  // 8 warps x 16 output features
    float acc[16][4];
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
    const int ntiles = N / 8;
#pragma unroll 1
    for (int kt = 0; kt < MLP_CHUNK / 16; ++kt) {
        uint32_t a[4];
        const bf16 *pa = sD + (m0 + g) * LDC + 16 * kt + 2 * t;
        a[0] = ld32(pa);
        a[1] = ld32(pa + 8 * LDC);
        a[2] = ld32(pa + 8);
        a[3] = ld32(pa + 8 * LDC + 8);
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) {
            if (nt < ntiles) {
                const bf16 *pb = sHp + (8 * nt + g) * LDC + 16 * kt + 2 * t;
                mma16816(acc[nt], a, ld32(pb), ld32(pb + 8));
            }
        }
    }
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
        if (nt < ntiles) {
            const int i = 8 * nt + 2 * t, o = m0 + g;
            out[offW + o * N + i] = acc[nt][0];
            out[offW + o * N + i + 1] = acc[nt][1];
            out[offW + (o + 8) * N + i] = acc[nt][2];
            out[offW + (o + 8) * N + i + 1] = acc[nt][3];
        }
    }
    if (threadIdx.x < H) {  // bias gradient: sum of dh over the chunk's rows
        float s = 0.0f;
        for (int r = 0; r < MLP_CHUNK; ++r) s += __bfloat162float(sD[threadIdx.x * LDC + r]);
        out[offB + threadIdx.x] = s;
    }
    if (L == 3) {  // output unit
        if (threadIdx.x >= H) {
            const int i = threadIdx.x - H;
            float s = 0.0f;
            for (int r = 0; r < MLP_CHUNK && r0 + r < B; ++r)
                s += dz[r0 + r] * __bfloat162float(h3[(size_t)(r0 + r) * H + i]);
            out[MLP_OFF_W4 + i] = s;
        }
        if (threadIdx.x == 0) {
            float s = 0.0f;
            for (int r = 0; r < MLP_CHUNK && r0 + r < B; ++r) s += dz[r0 + r];
            out[MLP_OFF_B4] = s;
        }
    }
}

// Sums the chunks' gradients, optionally applies Adam (lr > 0) to the FP32
// master weights, and refreshes the BF16 copies (row-major for the forward
// pass, transposed for the backward pass).
__global__ void mlp_update_kernel(int nchunks, const float *part, float *master, float *am, float *av, float lr,
                                  float beta1, float beta2, float eps, float bc1, float bc2, float *grad_out,
                                  bf16 *w1b, bf16 *w2b, bf16 *w3b, bf16 *w2t, bf16 *w3t)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= MLP_NPARAM) return;
    float gsum = 0.0f;
    for (int c = 0; c < nchunks; ++c) gsum += part[(size_t)c * MLP_NPARAM + i];
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
    if (i < MLP_OFF_B1) {
        w1b[i - MLP_OFF_W1] = wb;
    } else if (i >= MLP_OFF_W2 && i < MLP_OFF_B2) {
        const int k = i - MLP_OFF_W2, o = k / H, in = k % H;
        w2b[k] = wb;
        w2t[in * H + o] = wb;
    } else if (i >= MLP_OFF_W3 && i < MLP_OFF_B3) {
        const int k = i - MLP_OFF_W3, o = k / H, in = k % H;
        w3b[k] = wb;
        w3t[in * H + o] = wb;
    }
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

constexpr int kMaxBatch = 8192;
constexpr int kChunks = kMaxBatch / MLP_CHUNK;
constexpr int kFwdSmem = (H * IN + 2 * H * H) * 2 + (4 * H + 4) * 4;
constexpr int kBwdSmem = 2 * H * H * 2 + H * 4;
constexpr int kWgSmem = 2 * H * LDC * 2;

}  // namespace

struct smc_mlp {
    int device = 0;
    int n_in = 0;
    std::string err;
    cudaStream_t stream = nullptr;
    float *master = nullptr, *am = nullptr, *av = nullptr, *part = nullptr, *grad = nullptr;
    bf16 *w1b = nullptr, *w2b = nullptr, *w3b = nullptr, *w2t = nullptr, *w3t = nullptr;
    bf16 *xb = nullptr, *h1 = nullptr, *h2 = nullptr, *h3 = nullptr, *dh1 = nullptr, *dh2 = nullptr, *dh3 = nullptr;
    float *yb = nullptr, *z = nullptr, *dz = nullptr, *loss = nullptr;
    int *h_err = nullptr, *d_err = nullptr;  // inference wait gave up (mapped host memory)
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
                                                              0.f, 0.f, 1.f, 1.f, nullptr, m->w1b, m->w2b, m->w3b,
                                                              m->w2t, m->w3t);
    MCK(cudaGetLastError());
    return SMC_OK;
}

// forward (+ backward and per-chunk weight gradients when y is given) over the
// B rows already gathered into xb / yb
int pass(smc_mlp *m, int B, bool train, cudaStream_t s)
{
    const int blocks = (B + MLP_ROWS_FWD - 1) / MLP_ROWS_FWD;
    mlp_fwd_kernel<<<blocks, 128, kFwdSmem, s>>>(m->xb, B, m->w1b, m->w2b, m->w3b, m->master, m->z,
                                                 train ? m->h1 : nullptr, train ? m->h2 : nullptr,
                                                 train ? m->h3 : nullptr);
    MCK(cudaGetLastError());
    if (!train) return SMC_OK;
    mlp_bwd_kernel<<<blocks, 128, kBwdSmem, s>>>(m->z, m->yb, B, 1.0f / (float)B, m->h1, m->h2, m->h3, m->w2t,
                                                 m->w3t, m->master, m->dz, m->dh1, m->dh2, m->dh3, m->loss);
    MCK(cudaGetLastError());
    const dim3 wg((B + MLP_CHUNK - 1) / MLP_CHUNK, 3);
    mlp_wgrad_kernel<<<wg, 256, kWgSmem, s>>>(B, m->xb, m->h1, m->h2, m->h3, m->dh1, m->dh2, m->dh3, m->dz,
                                              m->part);
    MCK(cudaGetLastError());
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
    if (cudaMalloc((void **)&m->part, (size_t)kChunks * np * 4) != cudaSuccess) return fin(SMC_E_OOM);
    void **wb[] = {(void **)&m->w1b, (void **)&m->w2b, (void **)&m->w3b, (void **)&m->w2t, (void **)&m->w3t};
    for (void **p : wb)
        if (cudaMalloc(p, (size_t)H * H * 2) != cudaSuccess) return fin(SMC_E_OOM);
    void **act[] = {(void **)&m->h1, (void **)&m->h2, (void **)&m->h3, (void **)&m->dh1, (void **)&m->dh2,
                    (void **)&m->dh3};
    for (void **p : act)
        if (cudaMalloc(p, (size_t)kMaxBatch * H * 2) != cudaSuccess) return fin(SMC_E_OOM);
    if (cudaMalloc((void **)&m->xb, (size_t)kMaxBatch * IN * 2) != cudaSuccess) return fin(SMC_E_OOM);
    void **vec[] = {(void **)&m->yb, (void **)&m->z, (void **)&m->dz};
    for (void **p : vec)
        if (cudaMalloc(p, (size_t)kMaxBatch * 4) != cudaSuccess) return fin(SMC_E_OOM);
    if (cudaMalloc((void **)&m->loss, 4096 * 4) != cudaSuccess) return fin(SMC_E_OOM);
    if (cudaHostAlloc((void **)&m->h_err, sizeof(int), cudaHostAllocMapped) != cudaSuccess) return fin(SMC_E_OOM);
    *m->h_err = 0;
    if (cudaHostGetDevicePointer((void **)&m->d_err, m->h_err, 0) != cudaSuccess) return fin(SMC_E_CUDA);
    const void *kern[] = {(const void *)mlp_fwd_kernel, (const void *)mlp_bwd_kernel,
                          (const void *)mlp_wgrad_kernel, (const void *)mlp_infer_kernel};
    const int smem[] = {kFwdSmem, kBwdSmem, kWgSmem, kTcSmem};
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
    void *ptrs[] = {m->master, m->am, m->av, m->part, m->grad, m->w1b, m->w2b, m->w3b, m->w2t, m->w3t,
                    m->xb, m->h1, m->h2, m->h3, m->dh1, m->dh2, m->dh3, m->yb, m->z, m->dz, m->loss};
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
    MCK(cudaSetDevice(m->device));
    cudaStream_t s = m->stream;
    mlp_gather_kernel<<<(n + 127) / 128, 128, 0, s>>>(x, y, (uint64_t)n, m->n_in, n, 0, 0, 0, 0, m->xb, m->yb);
    MCK(cudaGetLastError());
    MCK(cudaMemsetAsync(m->loss, 0, 4, s));
    int rc = pass(m, n, true, s);
    if (rc) return rc;
    const int nch = (n + MLP_CHUNK - 1) / MLP_CHUNK;
    mlp_update_kernel<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(nch, m->part, m->master, m->am, m->av, 0.0f, 0.f,
                                                              0.f, 0.f, 1.f, 1.f, m->grad, m->w1b, m->w2b,
                                                              m->w3b, m->w2t, m->w3t);
    MCK(cudaGetLastError());
    MCK(cudaMemcpyAsync(grad_host, m->grad, (size_t)MLP_NPARAM * 4, cudaMemcpyDeviceToHost, s));
    if (loss_host) MCK(cudaMemcpyAsync(loss_host, m->loss, 4, cudaMemcpyDeviceToHost, s));
    MCK(cudaStreamSynchronize(s));
    if (loss_host) *loss_host /= (float)n;
    return SMC_OK;
}

int smc_mlp_train(smc_mlp *m, const float *x, const float *y, uint64_t n, int epochs, int batch, float lr,
                  uint64_t seed, float *loss_host, void *stream)
{
    if (!m || !x || !y || n < 1 || epochs < 1 || epochs > 4096 || batch < 1 || batch > kMaxBatch || !(lr > 0.0f))
        return SMC_E_INVALID_ARG;
    MCK(cudaSetDevice(m->device));
    cudaStream_t s = stream ? (cudaStream_t)stream : m->stream;
    const uint64_t steps = (n + batch - 1) / (uint64_t)batch;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    MCK(cudaMemsetAsync(m->loss, 0, (size_t)epochs * 4, s));
    const int nch = (batch + MLP_CHUNK - 1) / MLP_CHUNK;
    for (int ep = 0; ep < epochs; ++ep) {
        for (uint64_t st = 0; st < steps; ++st) {
            const uint64_t step_id = (uint64_t)ep * steps + st;
            mlp_gather_kernel<<<(batch + 127) / 128, 128, 0, s>>>(x, y, n, m->n_in, batch, 0, 1, seed, step_id,
                                                                  m->xb, m->yb);
            MCK(cudaGetLastError());
            const int blocks = (batch + MLP_ROWS_FWD - 1) / MLP_ROWS_FWD;
            mlp_fwd_kernel<<<blocks, 128, kFwdSmem, s>>>(m->xb, batch, m->w1b, m->w2b, m->w3b, m->master, m->z,
                                                         m->h1, m->h2, m->h3);
            MCK(cudaGetLastError());
            mlp_bwd_kernel<<<blocks, 128, kBwdSmem, s>>>(m->z, m->yb, batch, 1.0f / (float)batch, m->h1, m->h2,
                                                         m->h3, m->w2t, m->w3t, m->master, m->dz, m->dh1, m->dh2,
                                                         m->dh3, m->loss + ep);
            MCK(cudaGetLastError());
            mlp_wgrad_kernel<<<dim3(nch, 3), 256, kWgSmem, s>>>(batch, m->xb, m->h1, m->h2, m->h3, m->dh1,
                                                                  m->dh2, m->dh3, m->dz, m->part);
            MCK(cudaGetLastError());
            ++m->adam_t;
            const float bc1 = 1.0f - std::pow(b1, (float)m->adam_t), bc2 = 1.0f - std::pow(b2, (float)m->adam_t);
            mlp_update_kernel<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(nch, m->part, m->master, m->am, m->av, lr,
                                                                      b1, b2, eps, bc1, bc2, nullptr, m->w1b,
                                                                      m->w2b, m->w3b, m->w2t, m->w3t);
            MCK(cudaGetLastError());
        }
    }
    if (loss_host) {
        MCK(cudaMemcpyAsync(loss_host, m->loss, (size_t)epochs * 4, cudaMemcpyDeviceToHost, s));
        MCK(cudaStreamSynchronize(s));
        for (int ep = 0; ep < epochs; ++ep) loss_host[ep] /= (float)(steps * (uint64_t)batch);
    }
    return SMC_OK;
}

int smc_mlp_predict_masked(smc_mlp *m, const float *x, uint64_t n, const uint8_t *skip, float *g, void *stream)
{
    if (!m || (n && (!x || !g))) return SMC_E_INVALID_ARG;
    if (*m->h_err)
        return mfail(m, SMC_E_CUDA, *m->h_err == 2 ? "an earlier inference launch gave up waiting for the tensor "
                                                     "cores and released tensor memory without their completion"
                                                   : "an earlier inference launch gave up waiting for the tensor cores");
    if (n == 0) return SMC_OK;
    MCK(cudaSetDevice(m->device));
    cudaStream_t s = stream ? (cudaStream_t)stream : m->stream;
    int dev_sm = 0;
    MCK(cudaDeviceGetAttribute(&dev_sm, cudaDevAttrMultiProcessorCount, m->device));
    // one CTA per SM (its shared memory rules out a second, which its
    // allocation of the whole tensor memory requires)
    const uint64_t tiles = (n + kTcRows - 1) / kTcRows;
    const uint64_t want = (tiles + kTcGroups - 1) / kTcGroups;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)dev_sm));
    mlp_infer_kernel<<<grid, kTcThreads, kTcSmem, s>>>(x, n, m->n_in, skip, m->w1b, m->w2b, m->w3b, m->master, g,
                                                       m->d_err);
    MCK(cudaGetLastError());
    return SMC_OK;
}

int smc_mlp_predict(smc_mlp *m, const float *x, uint64_t n, float *g, void *stream)
{
    return smc_mlp_predict_masked(m, x, n, nullptr, g, stream);
}

}  // extern "C"
