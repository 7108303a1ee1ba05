// smc_mlp_train.cuh -- one training step of the surrogate network on the
// fifth-generation tensor cores, fused into one kernel (included by
// smc_mlp.cu, inside its anonymous namespace, after the tcgen05 helpers).
//
// A step is this kernel and the Adam update (mlp_update_kernel), which sums
// the kernel's partial gradients.  The kernel runs one CTA per SM,
// persistent over the minibatch's 128-row tiles.  Per tile every activation
// and delta stays in shared memory and every product runs on tcgen05 (BF16
// operands, FP32 accumulators in tensor memory):
//
//   gather  X  = the tile's rows of x (BF16, zero-padded to 16 features)
//   forward h1 = relu(X W1^T + b1), h2, h3 the same (bias, ReLU, rounding in
//           the epilogue), z = h3 . w4 + b4 and dz = (sigmoid(z) - y) / B
//           on the CUDA cores, d3 = dz w4 [h3 > 0]
//   back    d2 = (d3 W3) [h2 > 0], d1 = (d2 W2) [h1 > 0]
//   grads   dW3 += d3^T h2, dW2 += d2^T h1, dW1 += d1^T X, db_l += d_l^T 1,
//           dw4 += h3^T dz  (the batch rows as the contraction index)
//
// A tensor-memory accumulator holds each layer's pre-activations (columns
// 0-127); the weight gradients accumulate across the CTA's tiles in columns
// 128-415, and at the end the CTA writes them as its partial gradient.
// Saved operands are read back as MN-major operands (smc_tc.h): an
// activation tile stored rows x features for the next layer serves as the
// features x rows operand of a weight gradient, and a weight matrix staged
// for the forward product as its own transpose.  Deltas overwrite
// activations once the products that read them have completed.

constexpr int kStWG = 2;                        // warpgroups: each takes 128 / kStWG columns of an epilogue
constexpr int kStThreads = 128 * kStWG;
constexpr int kStCols = H / kStWG;              // epilogue columns per thread
constexpr int kTileX = kTcRows * IN * 2;        // [128][16] BF16, 4 KB
constexpr int kTileH = kTcRows * H * 2;         // [128][128] BF16, 32 KB
constexpr int kTileN16 = 16 * kTcRows * 2;      // [16][128] BF16, 4 KB (N = 16 operand, K = the rows)
// shared memory
constexpr int kStW1 = 0;
constexpr int kStW2 = kStW1 + H * IN * 2;
constexpr int kStW3 = kStW2 + H * H * 2;
constexpr int kStX = kStW3 + H * H * 2;         // two input tiles (the next tile's is written early)
constexpr int kStH1 = kStX + 2 * kTileX;
constexpr int kStH2 = kStH1 + kTileH;
constexpr int kStH3 = kStH2 + kTileH;           // h3, then d2
constexpr int kStD3 = kStH3 + kTileH;           // d3, then d1
constexpr int kStDz = kStD3 + kTileH;           // rows 3, 4: dz high and low parts; other rows 0
constexpr int kStOnes = kStDz + kTileN16;       // three tiles: row j of tile j is ones (j = 0, 1, 2)
constexpr int kStVec = kStOnes + 3 * kTileN16;  // FP32 b1, b2, b3, w4
constexpr int kStZp = kStVec + 4 * H * 4;       // FP32 [kStWG][128]: partial z per row
constexpr int kStBar = kStZp + kStWG * kTcRows * 4;
constexpr int kStSmem = kStBar + 8 + 8 + 8;     // products' mbarrier, weights' mbarrier, tensor-memory address
// tensor-memory columns
constexpr uint32_t kStAcc = 0;                  // a layer's pre-activations or pre-masked deltas
constexpr uint32_t kStDW2 = 128, kStDW3 = 256, kStDW1 = 384;
constexpr uint32_t kStBG = 400;                 // db1, db2, db3, dw4 (high), dw4 (low) in columns 400-404
constexpr int kStGradCols = 288;                // columns 128-415, read in 9 loads of 32
static_assert(kStSmem <= 227 * 1024, "shared memory per CTA");
static_assert(2 * (kStSmem + 1024) > 228 * 1024, "one CTA per SM (it takes the whole tensor memory)");
static_assert(kStBar % 8 == 0, "mbarrier alignment");
static_assert(kStCols % 32 == 0, "epilogue columns");
static_assert(128 + kStGradCols <= (int)kTcCols, "accumulator columns");

__device__ __forceinline__ uint64_t splitmix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

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

// Where the training rows come from: batch row i is row base + i of x (a
// gradient over given rows) or, when sample != 0, row hash(seed, step, i)
// mod n of x (a minibatch drawn with replacement; step = *step_ctr, which
// the update kernel advances).  Rows i >= B are padding (zero features,
// zero output delta).
struct StepRows {
    const float *x, *y;
    uint64_t n;
    int n_in, B;
    uint64_t base;
    int sample;
    uint64_t seed;
    const unsigned long long *step_ctr;
};

// this thread's part of row i of the batch: features 8c .. 8c + 7 (none
// for c >= 2) and the target; valid: a row of the batch, not padding
__device__ __forceinline__ void gather_row(const StepRows &rs, uint64_t step, uint64_t i, int c, float (&f)[8],
                                           float &yv, bool &valid)
{
    valid = i < (uint64_t)rs.B;
    uint64_t r = 0;
    if (valid) {
        r = rs.sample ? splitmix64(rs.seed ^ splitmix64(step * 0x100000001ull + i)) % rs.n : rs.base + i;
        valid = r < rs.n;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int col = 8 * c + k;
        f[k] = (valid && c < 2 && col < rs.n_in) ? rs.x[r * rs.n_in + col] : 0.0f;
    }
    yv = valid ? rs.y[r] : 0.0f;
}

// a CTA's partial gradient: every parameter, at part + blockIdx.x * kPartStride
// (a multiple of 4 floats, so that the rows of W1, W2, W3 start 16-byte aligned)
constexpr int kPartStride = (MLP_NPARAM + 31) / 32 * 32;
static_assert(MLP_OFF_W2 % 4 == 0 && MLP_OFF_W3 % 4 == 0 && MLP_OFF_W1 % 4 == 0, "16-byte aligned weight rows");

// One training step over the B rows of rs: the loss sum goes to *loss_acc,
// this CTA's partial gradient (every parameter) to part + blockIdx.x * kPartStride.  With
// adam_t set, CTA 0 advances *adam_t (the update kernel after this one reads
// it).  A tensor-core wait that gives up sets *err (2 if the products still
// in flight never completed) and the CTA writes no partial gradient.
__global__ void __launch_bounds__(kStThreads, 1)
    mlp_train_step_kernel(StepRows rs, float inv_b, const bf16 *w1b, const bf16 *w2b, const bf16 *w3b,
                          const float *master, float *part, float *loss_acc, unsigned long long *adam_t, int *err)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t *barp = reinterpret_cast<uint64_t *>(sm + kStBar);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + kStBar + 16);
    const uint32_t bar = smem_u32(barp), bar_w = smem_u32(barp + 1);
    const int tid = threadIdx.x, warp = tid >> 5, c = tid >> 7, r = tid & 127;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_w) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        stage_weights(smem_u32(sm + kStW1), w1b, w2b, w3b, bar_w);
        if (adam_t && blockIdx.x == 0) *adam_t += 1ull;
    }
    float *vec = reinterpret_cast<float *>(sm + kStVec);  // b1, b2, b3, w4
    if (tid < H) {
        const float v0 = master[MLP_OFF_B1 + tid], v1 = master[MLP_OFF_B2 + tid], v2 = master[MLP_OFF_B3 + tid],
                    v3 = master[MLP_OFF_W4 + tid];
        vec[tid] = v0;
        vec[H + tid] = v1;
        vec[2 * H + tid] = v2;
        vec[3 * H + tid] = v3;
    }
    const float b4 = master[MLP_OFF_B4];
    {   // the N = 16 tiles: dz (rows 3, 4 written per tile) zero, ones tile t with row t of ones
        const uint32_t one2 = pack_bf16x2(__float2bfloat16_rn(1.0f), __float2bfloat16_rn(1.0f));
        const uint4 z4 = make_uint4(0u, 0u, 0u, 0u), o4 = make_uint4(one2, one2, one2, one2);
        for (int i = tid; i < 16 * (kTcRows / 8); i += blockDim.x) {
            const int j = i / (kTcRows / 8), kg = i % (kTcRows / 8);
            const int off = tc_core_offset(j, kg, kTcRows);
            *reinterpret_cast<uint4 *>(sm + kStDz + off) = z4;
#pragma unroll
            for (int t = 0; t < 3; ++t) *reinterpret_cast<uint4 *>(sm + kStOnes + t * kTileN16 + off) = j == t ? o4 : z4;
        }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t t_lane = tmem + ((uint32_t)(32 * (warp & 3)) << 16);  // this warp's 32 lanes
    // the weights' copies (bounded wait; a CTA that gives up computes nothing)
    const bool w_failed = __syncthreads_or(!tc_wait(bar_w, 0));
    const uint32_t aW1 = smem_u32(sm + kStW1), aW2 = smem_u32(sm + kStW2), aW3 = smem_u32(sm + kStW3);
    const uint32_t aH1 = smem_u32(sm + kStH1), aH2 = smem_u32(sm + kStH2), aH3 = smem_u32(sm + kStH3);
    const uint32_t aD3 = smem_u32(sm + kStD3), aDz = smem_u32(sm + kStDz), aOnes = smem_u32(sm + kStOnes);
    const uint32_t lbo_h = tc_mn_lbo(H), sbo_h = tc_sbo(H);
    const uint64_t step = rs.step_ctr ? (uint64_t)*rs.step_ctr : 0;
    const uint64_t tiles = ((uint64_t)rs.B + kTcRows - 1) / kTcRows;
    uint32_t phase = 0;
    bool failed = w_failed;
    int count = 0;
    float loss = 0.0f, db4 = 0.0f;

    // all threads wait for the step's mbarrier; false (in every thread) if
    // any thread's wait gave up
    bool own_ok = true;  // this thread's last wait
    auto wait_all = [&]() -> bool {
        own_ok = tc_wait(bar, phase);
        phase ^= 1;
        return !__syncthreads_or(!own_ok);
    };
    // operands written by the threads -> visible to the tensor core; this
    // thread's tensor-memory reads complete before the next products
    auto sync_issue = [&]() {
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
    };
    // this thread's epilogue columns of the accumulator, two loads of 32 in
    // flight: fn(q, v) for q = 0 .. kStCols / 32 - 1 (columns c * kStCols + 32 q ...)
    auto acc_chunks = [&](auto &&fn) {
        uint32_t va[32], vb[32];
        const uint32_t base = t_lane + kStAcc + c * kStCols;
        tc_load32_async(base, va);
        tc_wait_ld(va);
#pragma unroll
        for (int q = 0; q < kStCols / 32; q += 2) {
            if (q + 1 < kStCols / 32) tc_load32_async(base + 32 * (q + 1), vb);
            fn(q, va);
            if (q + 1 < kStCols / 32) {
                tc_wait_ld(vb);
                if (q + 2 < kStCols / 32) tc_load32_async(base + 32 * (q + 2), va);
                fn(q + 1, vb);
                if (q + 2 < kStCols / 32) tc_wait_ld(va);
            }
        }
    };
    // h = relu(acc + bias) in BF16 -> dst (rows x 128, K-major)
    auto epi_hidden = [&](unsigned char *dst, const float *bias) {
        acc_chunks([&](int q, const uint32_t (&v)[32]) {
            const int col0 = c * kStCols + 32 * q;
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                uint32_t w[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int k = 8 * g + 2 * j;
                    w[j] = relu_pack2(__float_as_uint(__uint_as_float(v[k]) + bias[col0 + k]),
                                      __float_as_uint(__uint_as_float(v[k + 1]) + bias[col0 + k + 1]));
                }
                *reinterpret_cast<uint4 *>(dst + tc_core_offset(r, col0 / 8 + g, H)) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        });
    };
    // d = acc [mask > 0] in BF16 -> dst
    auto epi_delta = [&](const unsigned char *mask, unsigned char *dst) {
        acc_chunks([&](int q, const uint32_t (&v)[32]) {
            const int col0 = c * kStCols + 32 * q;
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                float f[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) f[j] = __uint_as_float(v[8 * g + j]);
                const int off = tc_core_offset(r, col0 / 8 + g, H);
                *reinterpret_cast<uint4 *>(dst + off) = mask_pack8(*reinterpret_cast<const uint4 *>(mask + off), f);
            }
        });
    };

    float f[8], yv = 0.0f;
    bool valid = false;
    uint64_t tile = failed ? tiles : blockIdx.x;
    if (tile < tiles) gather_row(rs, step, tile * kTcRows + r, c, f, yv, valid);
    int xb = 0;
    for (; tile < tiles; tile += gridDim.x, xb ^= 1) {
        const bool first = count == 0;
        unsigned char *X = sm + kStX + xb * kTileX;
        const uint32_t aX = smem_u32(X);
        if (c < 2) {
            const uint4 v = make_uint4(pack2(f[0], f[1]), pack2(f[2], f[3]), pack2(f[4], f[5]), pack2(f[6], f[7]));
            *reinterpret_cast<uint4 *>(X + tc_core_offset(r, c, IN)) = v;
        }
        const float y_t = yv;
        const bool valid_t = valid;
        if (tile + gridDim.x < tiles) gather_row(rs, step, (tile + gridDim.x) * kTcRows + r, c, f, yv, valid);

        // forward: h1, h2, h3
        sync_issue();
        if (tid == 0) {
            tc_fence_after();
            tc_mma(tmem + kStAcc, tc_desc(aX, kTcLbo, tc_sbo(IN)), tc_desc(aW1, kTcLbo, tc_sbo(IN)), tc_idesc(H), 0);
            tc_commit(bar);
        }
        if (!wait_all()) { failed = true; break; }
        tc_fence_after();
        epi_hidden(sm + kStH1, vec);
        for (int layer = 0; layer < 2; ++layer) {
            const uint32_t aA = layer == 0 ? aH1 : aH2, aW = layer == 0 ? aW2 : aW3;
            sync_issue();
            if (tid == 0) {
                tc_fence_after();
#pragma unroll
                for (int s = 0; s < H / 16; ++s)
                    tc_mma(tmem + kStAcc, tc_desc(aA + 256 * s, kTcLbo, sbo_h), tc_desc(aW + 256 * s, kTcLbo, sbo_h),
                           tc_idesc(H), s > 0);
                tc_commit(bar);
            }
            if (!wait_all()) { failed = true; break; }
            tc_fence_after();
            if (layer == 0) epi_hidden(sm + kStH2, vec + H);
        }
        if (failed) break;

        // h3 = relu(acc + b3), z = h3 . w4 + b4, dz, d3 = dz w4 [h3 > 0]
        {
            uint32_t hw[kStCols / 2];  // this thread's h3 values, packed BF16 pairs
            float zp = 0.0f;
            const float *b3 = vec + 2 * H, *w4 = vec + 3 * H;
            acc_chunks([&](int q, const uint32_t (&v)[32]) {
                const int col0 = c * kStCols + 32 * q;
#pragma unroll
                for (int g = 0; g < 4; ++g) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int k = 8 * g + 2 * j;
                        const uint32_t w = relu_pack2(__float_as_uint(__uint_as_float(v[k]) + b3[col0 + k]),
                                                      __float_as_uint(__uint_as_float(v[k + 1]) + b3[col0 + k + 1]));
                        hw[16 * q + 4 * g + j] = w;
                        const float2 h = unpack2(w);
                        zp = fmaf(h.x, w4[col0 + k], zp);
                        zp = fmaf(h.y, w4[col0 + k + 1], zp);
                    }
                    const int o = 16 * q + 4 * g;
                    *reinterpret_cast<uint4 *>(sm + kStH3 + tc_core_offset(r, col0 / 8 + g, H)) =
                        make_uint4(hw[o], hw[o + 1], hw[o + 2], hw[o + 3]);
                }
            });
            float *zpart = reinterpret_cast<float *>(sm + kStZp);
            zpart[c * kTcRows + r] = zp;
            __syncthreads();
            float z = b4;
#pragma unroll
            for (int cc = 0; cc < kStWG; ++cc) z += zpart[cc * kTcRows + r];
            float dz = 0.0f;
            if (valid_t) {
                dz = (1.0f / (1.0f + expf(-z)) - y_t) * inv_b;
                if (c == 0) loss += fmaxf(z, 0.0f) - z * y_t + log1pf(expf(-fabsf(z)));
            }
            if (c == 0) {
                db4 += dz;
                *tc_elem(sm + kStDz, 3, r, kTcRows) = bf16_hi(dz);
                *tc_elem(sm + kStDz, 4, r, kTcRows) = bf16_lo(dz);
            }
#pragma unroll
            for (int g = 0; g < kStCols / 8; ++g) {
                const int col0 = c * kStCols + 8 * g;
                float v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = dz * w4[col0 + j];
                const uint4 hv = make_uint4(hw[4 * g], hw[4 * g + 1], hw[4 * g + 2], hw[4 * g + 3]);
                *reinterpret_cast<uint4 *>(sm + kStD3 + tc_core_offset(r, col0 / 8, H)) = mask_pack8(hv, v);
            }
        }

        // dw4 += h3^T dz, db3 += d3^T 1, acc = d3 W3 (committed); dW3 += d3^T h2
        sync_issue();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t i16 = tc_idesc_bf16_t(128, 16, true, false);
#pragma unroll
            for (int s = 0; s < kTcRows / 16; ++s)
                tc_mma(tmem + kStBG, tc_desc(aH3 + 2 * lbo_h * s, lbo_h, kTcMnSbo),
                       tc_desc(aDz + 256 * s, kTcLbo, tc_sbo(kTcRows)), i16, !(first && s == 0));
#pragma unroll
            for (int s = 0; s < kTcRows / 16; ++s)
                tc_mma(tmem + kStBG, tc_desc(aD3 + 2 * lbo_h * s, lbo_h, kTcMnSbo),
                       tc_desc(aOnes + 2 * kTileN16 + 256 * s, kTcLbo, tc_sbo(kTcRows)), i16, 1);
#pragma unroll
            for (int s = 0; s < H / 16; ++s)
                tc_mma(tmem + kStAcc, tc_desc(aD3 + 256 * s, kTcLbo, sbo_h), tc_desc(aW3 + 2 * lbo_h * s, lbo_h, kTcMnSbo),
                       tc_idesc_bf16_t(128, H, false, true), s > 0);
            tc_commit(bar);
#pragma unroll
            for (int s = 0; s < kTcRows / 16; ++s)
                tc_mma(tmem + kStDW3, tc_desc(aD3 + 2 * lbo_h * s, lbo_h, kTcMnSbo),
                       tc_desc(aH2 + 2 * lbo_h * s, lbo_h, kTcMnSbo), tc_idesc_bf16_t(128, H, true, true),
                       !(first && s == 0));
        }
        if (!wait_all()) { failed = true; break; }
        tc_fence_after();
        epi_delta(sm + kStH2, sm + kStH3);  // d2 over h3

        // db2 += d2^T 1, acc = d2 W2 (committed); dW2 += d2^T h1
        sync_issue();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int s = 0; s < kTcRows / 16; ++s)
                tc_mma(tmem + kStBG, tc_desc(aH3 + 2 * lbo_h * s, lbo_h, kTcMnSbo),
                       tc_desc(aOnes + kTileN16 + 256 * s, kTcLbo, tc_sbo(kTcRows)),
                       tc_idesc_bf16_t(128, 16, true, false), 1);
#pragma unroll
            for (int s = 0; s < H / 16; ++s)
                tc_mma(tmem + kStAcc, tc_desc(aH3 + 256 * s, kTcLbo, sbo_h), tc_desc(aW2 + 2 * lbo_h * s, lbo_h, kTcMnSbo),
                       tc_idesc_bf16_t(128, H, false, true), s > 0);
            tc_commit(bar);
#pragma unroll
            for (int s = 0; s < kTcRows / 16; ++s)
                tc_mma(tmem + kStDW2, tc_desc(aH3 + 2 * lbo_h * s, lbo_h, kTcMnSbo),
                       tc_desc(aH1 + 2 * lbo_h * s, lbo_h, kTcMnSbo), tc_idesc_bf16_t(128, H, true, true),
                       !(first && s == 0));
        }
        if (!wait_all()) { failed = true; break; }
        tc_fence_after();
        epi_delta(sm + kStH1, sm + kStD3);  // d1 over d3

        // db1 += d1^T 1, dW1 += d1^T X (completed before the next tile's first product)
        sync_issue();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t lbo_x = tc_mn_lbo(IN);
#pragma unroll
            for (int s = 0; s < kTcRows / 16; ++s) {
                tc_mma(tmem + kStBG, tc_desc(aD3 + 2 * lbo_h * s, lbo_h, kTcMnSbo),
                       tc_desc(aOnes + 256 * s, kTcLbo, tc_sbo(kTcRows)), tc_idesc_bf16_t(128, 16, true, false), 1);
                tc_mma(tmem + kStDW1, tc_desc(aD3 + 2 * lbo_h * s, lbo_h, kTcMnSbo),
                       tc_desc(aX + 2 * lbo_x * s, lbo_x, kTcMnSbo), tc_idesc_bf16_t(128, 16, true, true),
                       !(first && s == 0));
            }
        }
        ++count;
    }
    // every product of the CTA complete before its accumulators are read
    if (!failed && count > 0) {
        sync_issue();
        if (tid == 0) {
            tc_fence_after();
            tc_commit(bar);
        }
        if (!wait_all()) failed = true;
        tc_fence_after();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        loss += __shfl_xor_sync(0xffffffffu, loss, o);
        db4 += __shfl_xor_sync(0xffffffffu, db4, o);
    }
    if (!failed) {
        if ((tid & 31) == 0 && loss != 0.0f) atomicAdd(loss_acc, loss);
        // the partial gradient: thread (r, c) holds accumulator lane r, i.e.
        // output feature o = r of every weight gradient, and writes the
        // column chunks k = c, c + kStWG, ... of the 9 chunks of 32 straight
        // from its registers (a chunk of dW2 or dW3 is 32 consecutive
        // entries of row o)
        float *out = part + (size_t)blockIdx.x * kPartStride;
        const int o = r;
        for (int k = c; k < kStGradCols / 32; k += kStWG) {
            const int c0 = 128 + 32 * k;
            uint32_t v[32];
            if (count > 0) {
                tc_load32_async(t_lane + c0, v);
                tc_wait_ld(v);
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = 0u;
            }
            if (c0 < 384) {  // dW2 (columns 128-255) or dW3 (256-383)
                float4 *dst = reinterpret_cast<float4 *>(
                    out + (c0 < 256 ? MLP_OFF_W2 + o * H + (c0 - 128) : MLP_OFF_W3 + o * H + (c0 - 256)));
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    dst[q] = make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                                         __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
            } else {  // dW1 (384-399), db1, db2, db3 (400-402), dw4 = high + low (403, 404)
                float4 *dst = reinterpret_cast<float4 *>(out + MLP_OFF_W1 + o * IN);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    dst[q] = make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                                         __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
                out[MLP_OFF_B1 + o] = __uint_as_float(v[16]);
                out[MLP_OFF_B2 + o] = __uint_as_float(v[17]);
                out[MLP_OFF_B3 + o] = __uint_as_float(v[18]);
                out[MLP_OFF_W4 + o] = __uint_as_float(v[19]) + __uint_as_float(v[20]);
            }
        }
        float *red = reinterpret_cast<float *>(sm + kStZp);
        __syncthreads();
        if ((tid & 31) == 0) red[warp] = db4;
        __syncthreads();
        if (tid == 0) {
            float s = 0.0f;
            for (int w = 0; w < 4; ++w) s += red[w];  // warps 0-3 hold the rows' dz (warpgroup 0)
            out[MLP_OFF_B4] = s;
        }
    } else if (w_failed) {
        if (tid == 0) {  // no products were issued; the copies must land before the CTA exits
            atomicExch(err, 1);
            bool drained = false;
            for (int k = 0; k < 4 && !drained; ++k) drained = tc_wait(bar_w, 0);
            if (!drained) atomicExch(err, 2);
        }
    } else if (tid == 0) {
        // a wait gave up: wait (bounded) for the products in flight, the last
        // committed ones (unless this thread saw them complete) and then any
        // issued after them, before the tensor memory is released
        atomicExch(err, 1);
        bool drained = own_ok;
        for (int k = 0; k < 4 && !drained; ++k) drained = tc_wait(bar, phase ^ 1);
        if (drained) {
            tc_commit(bar);
            drained = false;
            for (int k = 0; k < 4 && !drained; ++k) drained = tc_wait(bar, phase);
        }
        if (!drained) atomicExch(err, 2);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
    }
}
