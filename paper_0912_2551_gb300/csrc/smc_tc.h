// smc_tc.h -- encodings for the fifth-generation tensor cores (tcgen05) used
// by the surrogate network's kernels: the shared-memory operand layout, the
// shared-memory matrix descriptor and the instruction descriptor.  Host and device constexpr functions, so that a host program
// can check them (tests/tc_encoding_check.cpp).
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define SMC_TC_HD __host__ __device__
#else
#define SMC_TC_HD
#endif

// K-major operand without swizzling: an R x K BF16 operand is stored as core
// matrices of 8 rows x 16 bytes (8 values along K), 128 contiguous bytes
// each; core matrix (r / 8, kg) starts at byte ((r / 8) * (K / 8) + kg) *
// 128, its row r % 8 at + (r % 8) * 16.  Neighbouring core matrices along K
// are therefore 128 bytes apart (the descriptor's leading byte offset) and
// neighbouring 8-row groups K * 16 bytes apart (its stride byte offset).
SMC_TC_HD constexpr int tc_core_offset(int r, int kg, int K)
{
    return ((r >> 3) * (K >> 3) + kg) * 128 + (r & 7) * 16;
}

// byte offset of element (r, k)
SMC_TC_HD constexpr int tc_elem_offset(int r, int k, int K) { return tc_core_offset(r, k >> 3, K) + (k & 7) * 2; }

constexpr uint32_t kTcLbo = 128;  // leading byte offset of the layout above
SMC_TC_HD constexpr uint32_t tc_sbo(int K) { return (uint32_t)K * 16; }  // its stride byte offset

// The same stored R x C tile read as an MN-major operand (the instruction
// descriptor's transpose bit set) whose MN index is the column c (C values)
// and whose K index is the row r: an MN-major core matrix is 8 rows along K
// of 16 bytes (8 values) along MN, which is exactly a stored core matrix;
// neighbouring core matrices along MN are 128 bytes apart (the descriptor's
// stride byte offset for MN-major operands), along K (8-row groups) C * 16
// bytes apart (its leading byte offset).  So the activations of a layer,
// stored rows x features for the next layer's product, serve unchanged as
// the features x rows operand of the weight gradients, and a weight matrix
// stored for the forward product serves as its own transpose.
constexpr uint32_t kTcMnSbo = 128;
SMC_TC_HD constexpr uint32_t tc_mn_lbo(int C) { return (uint32_t)C * 16; }

// shared-memory matrix descriptor: bits 0-13 start address >> 4, 16-29
// leading byte offset >> 4, 32-45 stride byte offset >> 4, 46-47 descriptor
// version (1), 49-51 base offset (0), 52 leading-offset mode (0: relative),
// 61-63 swizzle mode (0: none)
SMC_TC_HD constexpr uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of tcgen05.mma kind::f16 with BF16 A and B and an
// FP32 accumulator, both operands K-major, dense: bits 4-5 D format (1:
// F32), 7-9 A format (1: BF16), 10-12 B format (1: BF16), 13-14 negate A/B
// (0), 15-16 transpose A/B (0: K-major), 17-22 N >> 3, 24-28 M >> 4
SMC_TC_HD constexpr uint32_t tc_idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// the same with A and/or B MN-major (bit 15 transposes A, bit 16 B)
SMC_TC_HD constexpr uint32_t tc_idesc_bf16_t(int M, int N, bool a_mn, bool b_mn)
{
    return tc_idesc_bf16(M, N) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16);
}
