// Host check of the tcgen05 encodings of paper_0912_2551_gb300/csrc/smc_tc.h
// used by the surrogate's inference kernel:
//  * the K-major core-matrix layout is a bijection from an R x K BF16
//    operand onto its R * K * 2 bytes, each core matrix (8 rows x 8 values)
//    one aligned 128-byte block, with neighbours along K at the leading byte
//    offset and neighbouring 8-row groups at the stride byte offset that the
//    kernel passes in its descriptors;
//  * the shared-memory descriptor and the instruction descriptor, decoded
//    field by field at the bit positions the PTX ISA documents for tcgen05.
// Prints "ok" and exits 0 when every check holds.
#include <stdint.h>
#include <stdio.h>

#include <vector>

#include "smc_tc.h"

static int failures = 0;
#define CHECK(c)                                                         \
    do {                                                                 \
        if (!(c)) {                                                      \
            ++failures;                                                  \
            if (failures < 20) printf("FAIL %s:%d %s\n", __FILE__, __LINE__, #c); \
        }                                                                \
    } while (0)

static uint64_t field(uint64_t v, int lo, int width) { return (v >> lo) & ((1ull << width) - 1); }

static void check_layout(int R, int K)
{
    std::vector<int> hits((size_t)R * K * 2, 0);
    for (int r = 0; r < R; ++r)
        for (int k = 0; k < K; ++k) {
            const int off = tc_elem_offset(r, k, K);
            CHECK(off >= 0 && off + 1 < R * K * 2 && off % 2 == 0);
            if (off < 0 || off + 1 >= R * K * 2) continue;
            ++hits[off];
            ++hits[off + 1];
            // the element's core matrix is the aligned 128-byte block of
            // its 8-row group and 8-value chunk, its row 16 bytes within
            const int block = off / 128, in = off % 128;
            CHECK(block == (r / 8) * (K / 8) + k / 8);
            CHECK(in / 16 == r % 8 && (in % 16) / 2 == k % 8);
            // descriptor strides: next chunk along K, next 8-row group
            if (k + 8 < K) CHECK(tc_elem_offset(r, k + 8, K) - off == (int)kTcLbo);
            if (r + 8 < R) CHECK(tc_elem_offset(r + 8, k, K) - off == (int)tc_sbo(K));
            // MMA step s (K = 16 per instruction) starts 256 s bytes in
            if (k % 16 == 0 && r < 8 && r % 8 == 0) CHECK(tc_elem_offset(0, k, K) == 256 * (k / 16));
        }
    for (size_t i = 0; i < hits.size(); ++i) CHECK(hits[i] == 1);
}

// The stored R x C tile read MN-major (MN = column c, K = row r): element
// (r, c) lies in the MN-major core matrix (c / 8, r / 8) at row r % 8 (16
// bytes each) and position c % 8; core matrices along MN are kTcMnSbo
// apart, along K tc_mn_lbo(C) apart; an MMA step along K (16 rows) starts
// 2 * tc_mn_lbo(C) bytes further.
static void check_mn_view(int R, int C)
{
    for (int r = 0; r < R; ++r)
        for (int c = 0; c < C; ++c) {
            const int off = tc_elem_offset(r, c, C);
            const int expect = (c / 8) * (int)kTcMnSbo + (r / 8) * (int)tc_mn_lbo(C) + (r % 8) * 16 + (c % 8) * 2;
            CHECK(off == expect);
            if (r % 16 == 0) CHECK(tc_elem_offset(r, c, C) - tc_elem_offset(0, c, C) == (r / 16) * 2 * (int)tc_mn_lbo(C));
        }
}

static void check_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    const uint64_t d = tc_desc(saddr, lbo, sbo);
    CHECK(field(d, 0, 14) == (saddr >> 4));   // start address >> 4
    CHECK(field(d, 14, 2) == 0);
    CHECK(field(d, 16, 14) == (lbo >> 4));    // leading byte offset >> 4
    CHECK(field(d, 30, 2) == 0);
    CHECK(field(d, 32, 14) == (sbo >> 4));    // stride byte offset >> 4
    CHECK(field(d, 46, 2) == 1);              // descriptor version
    CHECK(field(d, 48, 1) == 0);
    CHECK(field(d, 49, 3) == 0);              // base offset
    CHECK(field(d, 52, 1) == 0);              // leading-offset mode: relative
    CHECK(field(d, 53, 8) == 0);
    CHECK(field(d, 61, 3) == 0);              // swizzle: none
}

static void check_idesc(int M, int N)
{
    const uint64_t d = tc_idesc_bf16(M, N);
    CHECK(field(d, 0, 2) == 0 && field(d, 2, 1) == 0);  // dense
    CHECK(field(d, 3, 1) == 0);                         // no saturation
    CHECK(field(d, 4, 2) == 1);                         // D: F32
    CHECK(field(d, 6, 1) == 0);
    CHECK(field(d, 7, 3) == 1);                         // A: BF16
    CHECK(field(d, 10, 3) == 1);                        // B: BF16
    CHECK(field(d, 13, 1) == 0 && field(d, 14, 1) == 0);  // no negation
    CHECK(field(d, 15, 1) == 0 && field(d, 16, 1) == 0);  // both K-major
    CHECK(field(d, 17, 6) == (uint64_t)(N >> 3));
    CHECK(field(d, 23, 1) == 0);
    CHECK(field(d, 24, 5) == (uint64_t)(M >> 4));
    CHECK(field(d, 29, 3) == 0);
    CHECK(field(d, 32, 32) == 0);
    for (int t = 0; t < 4; ++t) {  // transpose bits of MN-major operands
        const uint64_t dt = tc_idesc_bf16_t(M, N, t & 1, t & 2);
        CHECK(field(dt, 15, 1) == (uint64_t)(t & 1) && field(dt, 16, 1) == (uint64_t)((t >> 1) & 1));
        CHECK((dt & ~((1ull << 15) | (1ull << 16))) == d);
    }
}

int main()
{
    // operands of the kernel: features and bias/ones tiles (128 x 16),
    // weights and activations (128 x 128), the output unit's B (16 x 128)
    // and its bias tile (16 x 16)
    const int shapes[][2] = {{128, 16}, {128, 128}, {16, 128}, {16, 16}};
    for (const auto &sh : shapes) check_layout(sh[0], sh[1]);
    for (const auto &sh : shapes) check_mn_view(sh[0], sh[1]);
    for (uint32_t a : {0u, 16u, 0x1230u, 0x11000u, 0x3FFF0u})
        for (int K : {16, 128}) check_desc(a, kTcLbo, tc_sbo(K));
    for (int N : {16, 128, 256}) check_idesc(128, N);
    check_idesc(64, 64);
    if (failures) {
        printf("failures=%d\n", failures);
        return 1;
    }
    printf("ok\n");
    return 0;
}
