// smc_mlp_train.cuh -- the surrogate network's backward pass and weight
// gradients on the fifth-generation tensor cores (included by smc_mlp.cu,
// inside its anonymous namespace, after the forward kernel and the tcgen05
// helpers).
//
// A training step is: gather the minibatch (BF16 rows), the forward kernel
// (mlp_tc_forward<true>: logits and every layer's activations saved as
// 128-row tiles in the operand layout), the backward kernel below (output
// deltas and the hidden layers' deltas, saved the same way), the weight-
// gradient kernel below (one partial gradient per CTA) and the Adam update
// (which sums the partials).  Every product runs on tcgen05 with BF16
// operands and FP32 accumulators in tensor memory; the saved tiles are read
// back as MN-major operands (smc_tc.h), so no tile is ever transposed.

// ---------------------------------------------------------------------------
// Backward pass.  Per 128-row tile (kTcGroups pipelines per CTA, as in the
// forward kernel): dz = (sigmoid(z) - y) / B for the rows of the batch and 0
// beyond it, d3 = dz w4 [h3 > 0] on the CUDA cores, then d2 = (d3 W3)
// [h2 > 0] and d1 = (d2 W2) [h1 > 0] as MMAs with A = the delta tile
// (K-major, rows x features) and B = the weight matrix as staged for the
// forward product, read MN-major (its own transpose).  Deltas are rounded
// to BF16 and saved; the summed cross-entropy goes to *loss_acc.
constexpr int kBwSmW2 = 0;
constexpr int kBwSmW3 = kBwSmW2 + H * H * 2;
constexpr int kBwSmW4 = kBwSmW3 + H * H * 2;  // w4 in FP32
constexpr int kBwSmBar = kBwSmW4 + H * 4;
constexpr int kBwSmGroup = (kBwSmBar + 8 * kTcGroups + 4 + 1023) / 1024 * 1024;
constexpr int kBwSmem = kBwSmGroup + kTcGroups * kTileH;
static_assert(kBwSmBar % 8 == 0, "mbarrier alignment");
static_assert(kBwSmem <= 227 * 1024, "shared memory per CTA");
static_assert(2 * (kBwSmem + 1024) > 228 * 1024, "one CTA per SM (it takes the whole tensor memory)");

// 8 BF16 values of a saved activation row and 8 FP32 products: the products
// where the activation is positive, 0 elsewhere, rounded to BF16 and packed
__device__ __forceinline__ uint4 mask_pack8(const uint4 hv, const float (&v)[8])
{
    const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w};
    uint32_t o[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float2 h = unpack2(hw[j]);
        o[j] = pack2(h.x > 0.0f ? v[2 * j] : 0.0f, h.y > 0.0f ? v[2 * j + 1] : 0.0f);
    }
    return make_uint4(o[0], o[1], o[2], o[3]);
}

__global__ void __launch_bounds__(kTcThreads) mlp_train_bwd_kernel(const float *__restrict__ y, uint64_t n,
                                                                   float inv_b, const bf16 *w2b, const bf16 *w3b,
                                                                   const float *master, TrainTiles tt,
                                                                   float *loss_acc, int *err)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + kBwSmBar);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + kBwSmBar + 8 * kTcGroups);
    const int tid = threadIdx.x, warp = tid >> 5, grp = tid >> 7, gt = tid & 127;
    const int bid = 1 + grp;
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
    tc_stage_operand(sm + kBwSmW2, w2b, H, H);
    tc_stage_operand(sm + kBwSmW3, w3b, H, H);
    float *sw4 = reinterpret_cast<float *>(sm + kBwSmW4);
    for (int i = tid; i < H; i += blockDim.x) sw4[i] = master[MLP_OFF_W4 + i];
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t tacc = tmem + 128u * grp;
    const uint32_t t_row = tacc + ((uint32_t)(32 * (warp & 3)) << 16);
    unsigned char *act = sm + kBwSmGroup + grp * kTileH;
    const uint32_t bar = smem_u32(bars + grp), aAct = smem_u32(act);
    uint32_t phase = 0;
    bool failed = false;
    float loss = 0.0f;
    const uint64_t tiles = (n + kTcRows - 1) / kTcRows;
    for (uint64_t tile = (uint64_t)blockIdx.x * kTcGroups + grp; tile < tiles;
         tile += (uint64_t)gridDim.x * kTcGroups) {
        const uint64_t row = tile * kTcRows + gt;
        float dz = 0.0f;
        if (row < n) {
            const float zz = tt.z[row], yy = y[row];
            dz = (1.0f / (1.0f + expf(-zz)) - yy) * inv_b;
            loss += fmaxf(zz, 0.0f) - zz * yy + log1pf(expf(-fabsf(zz)));
        }
        tt.dz[row] = dz;
        {   // d3 = dz w4 [h3 > 0]
            const unsigned char *hg = tt.h3 + tile * kTileH;
            unsigned char *dg = tt.d3 + tile * kTileH;
#pragma unroll 4
            for (int kg = 0; kg < H / 8; ++kg) {
                float v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = dz * sw4[8 * kg + j];
                const uint4 w = mask_pack8(*reinterpret_cast<const uint4 *>(hg + tc_core_offset(gt, kg, H)), v);
                *reinterpret_cast<uint4 *>(act + tc_core_offset(gt, kg, H)) = w;
                *reinterpret_cast<uint4 *>(dg + tc_core_offset(gt, kg, H)) = w;
            }
        }
        for (int layer = 0; layer < 2; ++layer) {  // d2 through W3, then d1 through W2
            fence_async_smem();
            tc_fence_before();
            group_sync(bid);
            if (gt == 0) {
                tc_fence_after();
                const uint32_t aW = smem_u32(sm + (layer == 0 ? kBwSmW3 : kBwSmW2));
#pragma unroll
                for (int s = 0; s < H / 16; ++s)
                    tc_mma(tacc, tc_desc(aAct + 256 * s, kTcLbo, tc_sbo(H)),
                           tc_desc(aW + 2 * tc_mn_lbo(H) * s, tc_mn_lbo(H), kTcMnSbo), tc_idesc_bf16_t(128, H, false, true),
                           s > 0);
                tc_commit(bar);
            }
            const bool ok = tc_wait(bar, phase);
            phase ^= 1;
            if (group_or(bid, !ok)) {
                failed = true;
                break;
            }
            tc_fence_after();
            const unsigned char *hg = (layer == 0 ? tt.h2 : tt.h1) + tile * kTileH;
            unsigned char *dg = (layer == 0 ? tt.d2 : tt.d1) + tile * kTileH;
            for (int c = 0; c < H / 32; ++c) {
                uint32_t v[32];
                tc_load32_async(t_row + 32 * c, v);
                tc_wait_ld(v);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int kg = 4 * c + q;
                    float f[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) f[j] = __uint_as_float(v[8 * q + j]);
                    const uint4 w = mask_pack8(*reinterpret_cast<const uint4 *>(hg + tc_core_offset(gt, kg, H)), f);
                    if (layer == 0) *reinterpret_cast<uint4 *>(act + tc_core_offset(gt, kg, H)) = w;
                    *reinterpret_cast<uint4 *>(dg + tc_core_offset(gt, kg, H)) = w;
                }
            }
        }
        if (failed) {
            if (gt == 0) atomicExch(err, 1);
            break;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
    if ((tid & 31) == 0 && loss != 0.0f) atomicAdd(loss_acc, loss);
    // tensor memory is released once every product of this CTA has finished
    // (a pipeline that gave up waits again, bounded, as in the forward kernel)
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

// ---------------------------------------------------------------------------
// Weight gradients.  One CTA of 128 threads per SM, persistent over the
// tiles (tile = blockIdx.x, blockIdx.x + gridDim.x, ...).  Per tile its
// seven saved tiles are copied into shared memory (cp.async.bulk, completion
// on one mbarrier) and the products accumulate in tensor memory across the
// CTA's tiles, the batch rows as the contraction index K:
//   dW_l[o][i] += sum_r d_l[r][o] h_(l-1)[r][i]   A = d_l, B = h_(l-1), both MN-major
//   db_l[o]    += sum_r d_l[r][o]                 B = a K-major tile of ones
//   dw4[i]     += sum_r h3[r][i] dz[r]            A = h3 (MN-major), B = dz in BF16
//                                                 high and low parts (K-major)
// (h_0 = the input tile; dz beyond the batch is 0).  At the end each thread
// reads its accumulator lane (one output feature) and the CTA writes its
// partial gradient, every parameter, to part[blockIdx.x]; db4 = sum dz.
// Shared memory: the six 32 KB tiles first, then the input tile, dz, the
// ones and the barriers.  An MN-major operand at tile offset 4096 s reaches
// at most 32 KB into its tile; the allocation also covers 59,648 bytes past
// the last tile's start, so that every descriptor read stays inside it
// whatever the strides (it would if the two MN-major strides were read the
// other way round).
constexpr int kWgH1 = 0;
constexpr int kWgH2 = kWgH1 + kTileH;
constexpr int kWgH3 = kWgH2 + kTileH;
constexpr int kWgD1 = kWgH3 + kTileH;
constexpr int kWgD2 = kWgD1 + kTileH;
constexpr int kWgD3 = kWgD2 + kTileH;
constexpr int kWgX = kWgD3 + kTileH;
constexpr int kWgDz = kWgX + kTileX;               // [16][128] BF16: dz high, dz low, zeros
constexpr int kWgOnes = kWgDz + 16 * kTcRows * 2;  // [16][128] BF16 ones
constexpr int kWgBar = kWgOnes + 16 * kTcRows * 2;
constexpr int kWgSmemUsed = kWgBar + 2 * 8 + 16;
constexpr int kWgReach = kWgD3 + (kTcRows / 16 - 1) * 4096 + 15 * 2048 + 128 + 128;
constexpr int kWgSmem = kWgSmemUsed > kWgReach ? kWgSmemUsed : kWgReach;
constexpr uint32_t kWgCopyBytes = kTileX + 6 * kTileH;
// accumulator columns, each aligned to its width
constexpr uint32_t kColW2 = 0, kColW3 = 128, kColW1 = 256, kColB1 = 272, kColB2 = 288, kColB3 = 304, kColW4 = 320;
constexpr int kWgColsRead = 352;  // 11 loads of 32 columns cover all of them
static_assert(kWgSmem <= 227 * 1024, "shared memory per CTA");
static_assert(2 * (kWgSmem + 1024) > 228 * 1024, "one CTA per SM (it takes the whole tensor memory)");
static_assert(kWgColsRead <= (int)kTcCols, "accumulator columns");

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// parameter index of accumulator column col for output feature (lane) o;
// -1 for columns that are not read (the unused columns of the N = 16 products)
__device__ __forceinline__ int wgrad_param(int col, int o)
{
    if (col < 128) return MLP_OFF_W2 + o * H + col;
    if (col < 256) return MLP_OFF_W3 + o * H + (col - 128);
    if (col < 272) return MLP_OFF_W1 + o * IN + (col - 256);
    if (col == (int)kColB1) return MLP_OFF_B1 + o;
    if (col == (int)kColB2) return MLP_OFF_B2 + o;
    if (col == (int)kColB3) return MLP_OFF_B3 + o;
    return -1;  // w4: the sum of columns 320 and 321, written separately
}

__global__ void __launch_bounds__(128) mlp_train_wgrad_kernel(uint64_t n_tiles, TrainTiles tt, float *part, int *err)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + kWgBar);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + kWgBar + 16);
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    const uint32_t bar_ld = smem_u32(bars), bar_mma = smem_u32(bars + 1);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_ld) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_mma) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const bf16 zero = __float2bfloat16_rn(0.0f), one = __float2bfloat16_rn(1.0f);
    for (int i = tid; i < 16 * kTcRows; i += blockDim.x) {
        const int r = i / kTcRows, k = i % kTcRows;
        *tc_elem(sm + kWgDz, r, k, kTcRows) = zero;
        *tc_elem(sm + kWgOnes, r, k, kTcRows) = one;
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t s0 = smem_u32(sm);
    uint32_t ph_ld = 0, ph_mma = 0;
    bool failed = false, mma_pending = false, copy_pending = false;
    int count = 0;
    float db4 = 0.0f;
    for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        if (tid == 0) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_ld), "r"(kWgCopyBytes)
                         : "memory");
            bulk_g2s(s0 + kWgX, tt.x + tile * kTileX, kTileX, bar_ld);
            bulk_g2s(s0 + kWgH1, tt.h1 + tile * kTileH, kTileH, bar_ld);
            bulk_g2s(s0 + kWgH2, tt.h2 + tile * kTileH, kTileH, bar_ld);
            bulk_g2s(s0 + kWgH3, tt.h3 + tile * kTileH, kTileH, bar_ld);
            bulk_g2s(s0 + kWgD1, tt.d1 + tile * kTileH, kTileH, bar_ld);
            bulk_g2s(s0 + kWgD2, tt.d2 + tile * kTileH, kTileH, bar_ld);
            bulk_g2s(s0 + kWgD3, tt.d3 + tile * kTileH, kTileH, bar_ld);
        }
        const float dz = tt.dz[tile * kTcRows + tid];
        db4 += dz;
        *tc_elem(sm + kWgDz, 0, tid, kTcRows) = bf16_hi(dz);
        *tc_elem(sm + kWgDz, 1, tid, kTcRows) = bf16_lo(dz);
        fence_async_smem();
        copy_pending = true;
        const bool ok = tc_wait(bar_ld, ph_ld);
        ph_ld ^= 1;
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        copy_pending = false;
        if (tid == 0) {
            tc_fence_after();
#pragma unroll 1
            for (int s = 0; s < kTcRows / 16; ++s) {
                const uint32_t acc = (count > 0 || s > 0) ? 1u : 0u;
                const uint32_t kH = s * 2 * tc_mn_lbo(H), kX = s * 2 * tc_mn_lbo(IN), kK = 256u * s;
                const uint64_t d1 = tc_desc(s0 + kWgD1 + kH, tc_mn_lbo(H), kTcMnSbo);
                const uint64_t d2 = tc_desc(s0 + kWgD2 + kH, tc_mn_lbo(H), kTcMnSbo);
                const uint64_t d3 = tc_desc(s0 + kWgD3 + kH, tc_mn_lbo(H), kTcMnSbo);
                const uint64_t ones = tc_desc(s0 + kWgOnes + kK, kTcLbo, tc_sbo(kTcRows));
                tc_mma(tmem + kColW1, d1, tc_desc(s0 + kWgX + kX, tc_mn_lbo(IN), kTcMnSbo),
                       tc_idesc_bf16_t(128, 16, true, true), acc);
                tc_mma(tmem + kColB1, d1, ones, tc_idesc_bf16_t(128, 16, true, false), acc);
                tc_mma(tmem + kColW2, d2, tc_desc(s0 + kWgH1 + kH, tc_mn_lbo(H), kTcMnSbo),
                       tc_idesc_bf16_t(128, H, true, true), acc);
                tc_mma(tmem + kColB2, d2, ones, tc_idesc_bf16_t(128, 16, true, false), acc);
                tc_mma(tmem + kColW3, d3, tc_desc(s0 + kWgH2 + kH, tc_mn_lbo(H), kTcMnSbo),
                       tc_idesc_bf16_t(128, H, true, true), acc);
                tc_mma(tmem + kColB3, d3, ones, tc_idesc_bf16_t(128, 16, true, false), acc);
                tc_mma(tmem + kColW4, tc_desc(s0 + kWgH3 + kH, tc_mn_lbo(H), kTcMnSbo),
                       tc_desc(s0 + kWgDz + kK, kTcLbo, tc_sbo(kTcRows)), tc_idesc_bf16_t(128, 16, true, false), acc);
            }
            tc_commit(bar_mma);
        }
        mma_pending = true;
        const bool ok2 = tc_wait(bar_mma, ph_mma);
        ph_mma ^= 1;
        if (__syncthreads_or(!ok2)) {
            failed = true;
            break;
        }
        mma_pending = false;
        tc_fence_after();
        ++count;
    }
    float *out = part + (size_t)blockIdx.x * MLP_NPARAM;
    if (!failed) {
        // the accumulators through shared memory (the tiles are free now), so
        // that the partial gradient is written row by row, coalesced
        float *st = reinterpret_cast<float *>(sm);  // [128][33]
        const uint32_t t_row = tmem + ((uint32_t)(32 * warp) << 16);
        for (int c0 = 0; c0 < kWgColsRead; c0 += 32) {
            uint32_t v[32];
            if (count > 0) {
                tc_load32_async(t_row + c0, v);
                tc_wait_ld(v);
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = 0u;
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) st[tid * 33 + j] = __uint_as_float(v[j]);
            __syncthreads();
            for (int idx = tid; idx < 128 * 32; idx += blockDim.x) {
                const int o = idx / 32, j = idx % 32, col = c0 + j;
                const int q = wgrad_param(col, o);
                if (q >= 0) out[q] = st[o * 33 + j];
                if (col == (int)kColW4) out[MLP_OFF_W4 + o] = st[o * 33 + j] + st[o * 33 + j + 1];
            }
            __syncthreads();
        }
        float s = db4;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        float *red = reinterpret_cast<float *>(sm) + 128 * 33;
        if ((tid & 31) == 0) red[warp] = s;
        __syncthreads();
        if (tid == 0) out[MLP_OFF_B4] = red[0] + red[1] + red[2] + red[3];
    } else {
        if (tid == 0) atomicExch(err, 1);
        if (tid == 0 && (mma_pending || copy_pending)) {  // bounded wait for what is in flight
            const uint32_t b = mma_pending ? bar_mma : bar_ld, ph = mma_pending ? ph_mma : ph_ld;
            bool drained = false;
            for (int k = 0; k < 4 && !drained; ++k) drained = tc_wait(b, ph ^ 1);
            if (!drained) atomicExch(err, 2);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
    }
}
