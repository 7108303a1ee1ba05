// smc_fp64i.h -- binary64 logarithm and division evaluated on the integer
// pipes.
//
// GB300 executes FP64 arithmetic at 2 lane-operations per clock per SM (one
// 32-lane instruction occupies the SM's FP64 unit for 16 clocks), while its
// integer units retire 64 or more lane-operations per clock.  The FP64 SSA
// path spends most of its FP64 budget on two operations per event (Eq. 2a):
// ln u and the division by a_0.  Here both are computed from the bit
// patterns with 64-bit integer arithmetic:
//
//   fp64i_div(n, d)   n / d rounded to nearest-even: the same bits as the
//                     IEEE-754 division for every input (positive normal
//                     operands with a normal quotient on the integer path,
//                     everything else by the hardware division).
//   fp64i_log(u, tab) ln u with a table-driven reduction (Tang, ACM TOMS 16,
//                     1990) in 128-bit fixed point: error below 0.502 ulp.
//
// The header compiles for the device (nvcc, NVRTC) and for the host (gcc,
// through unsigned __int128), so the same code is checked on the CPU
// against the platform's arithmetic.
#pragma once
#include <stdint.h>

#if defined(__CUDACC_RTC__)
#define FP64I_HD __host__ __device__ __forceinline__
#elif defined(__CUDACC__)
#include <math.h>
#include <string.h>
#define FP64I_HD __host__ __device__ __forceinline__
#else
#include <math.h>
#include <string.h>
#define FP64I_HD static inline
#endif

// Log table: F_j = 0.75 + j/256 (j = 0..192), g_j = round(2^18 / (192 + j))
// so that G_j = g_j / 1024 ~ 1/F_j.  Layout in 64-bit words:
//   [0, 193)         high words of ln G_j x 2^117 (signed 128-bit)
//   [193, 386)       low words
//   [386], [387]     ln 2 x 2^117, high and low word
//   [388, ...)       g_j as 193 uint32 (97 words, the last half unused)
#define FP64I_LOG_N 193
#define FP64I_LOG_WORDS (388 + 97)
#define FP64I_LOG_BYTES (((FP64I_LOG_WORDS * 8) + 15) / 16 * 16)

FP64I_HD uint64_t fp64i_mulhi(uint64_t a, uint64_t b)
{
#if defined(__CUDA_ARCH__)
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

FP64I_HD int fp64i_clz(uint64_t a)  // a != 0
{
#if defined(__CUDA_ARCH__)
    return __clzll((long long)a);
#else
    return __builtin_clzll(a);
#endif
}

FP64I_HD uint64_t fp64i_bits(double x)
{
#if defined(__CUDA_ARCH__)
    return (uint64_t)__double_as_longlong(x);
#else
    uint64_t b;
    memcpy(&b, &x, 8);
    return b;
#endif
}

FP64I_HD double fp64i_from_bits(uint64_t b)
{
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)b);
#else
    double x;
    memcpy(&x, &b, 8);
    return x;
#endif
}

FP64I_HD float fp64i_rcp_approx(float f)  // about 1/f (f in [2^23, 2^24))
{
#if defined(__CUDA_ARCH__)
    return __fdividef(1.0f, f);
#else
    return 1.0f / f;
#endif
}

#define FP64I_FRAC 0x000FFFFFFFFFFFFFull
#define FP64I_ONE (1ull << 52)

// n / d, correctly rounded (nearest, ties to even).
FP64I_HD double fp64i_div(double n, double d)
{
    const uint64_t bn = fp64i_bits(n), bd = fp64i_bits(d);
    const uint32_t en = (uint32_t)(bn >> 52), ed = (uint32_t)(bd >> 52);  // sign bit included
    if (en - 1u >= 0x7FEu || ed - 1u >= 0x7FEu) return n / d;  // zero, subnormal, inf, nan, negative
    uint64_t mn = (bn & FP64I_FRAC) | FP64I_ONE;
    const uint64_t md = (bd & FP64I_FRAC) | FP64I_ONE;
    int e = (int)en - (int)ed + 1023;  // biased exponent of the quotient for mn >= md
    if (mn < md) {
        mn <<= 1;
        --e;
    }
    if (e < 1 || e > 2046) return n / d;  // subnormal or infinite quotient
    if (md == FP64I_ONE)                  // a power of two: exact
        return fp64i_from_bits(((uint64_t)e << 52) | (mn & FP64I_FRAC));
    // 1/delta for delta = md / 2^53 in (1/2, 1), as y = Y 2^-63 in (1, 2):
    // a single-precision seed (relative error below 2^-21), then two Newton
    // steps y <- y (2 - delta y) in 64-bit fixed point (error about 2^-62).
    const uint64_t D = md << 11;  // delta 2^64
    const float s = fp64i_rcp_approx((float)(uint32_t)(D >> 40)) * 16777216.0f;
    uint64_t Y;
    {
        uint32_t sb;
#if defined(__CUDA_ARCH__)
        sb = __float_as_uint(s);
#else
        memcpy(&sb, &s, 4);
#endif
        // s in [1, 2]: its 24-bit significand scaled to 2^63; s = 2 saturates
        Y = (sb >= 0x40000000u) ? ~0ull : (((uint64_t)((sb & 0x7FFFFFu) | 0x800000u)) << 40);
    }
    for (int it = 0; it < 2; ++it) {
        // W = (2 - delta y) 2^63 = high word of 2^128 - D Y
        const uint64_t pl = D * Y, ph = fp64i_mulhi(D, Y);
        const uint64_t W = ~ph + (pl == 0);
        // Y <- Y W 2^-63
        const uint64_t ql = Y * W, qh = fp64i_mulhi(Y, W);
        Y = (qh << 1) | (ql >> 63);
    }
    // Qt = floor(mn 2^53 / md), in [2^53, 2^54): estimate mn Y 2^-63 (off by
    // at most 2), then the exact remainder fixes it
    uint64_t qt = (fp64i_mulhi(mn, Y) << 1) | ((mn * Y) >> 63);
    int64_t rem = (int64_t)((mn << 53) - qt * md);
    while (rem < 0) {
        --qt;
        rem += (int64_t)md;
    }
    while (rem >= (int64_t)md) {
        ++qt;
        rem -= (int64_t)md;
    }
    uint64_t q = qt >> 1;
    q += (qt & 1u) & (uint64_t)((rem != 0) | (int)(q & 1u));
    if (q >> 53) {  // rounded up to 2: next binade
        q >>= 1;
        if (++e > 2046) return n / d;
    }
    return fp64i_from_bits(((uint64_t)e << 52) | (q & FP64I_FRAC));
}

// ln u.  u = 2^k m' with m' in [0.75, 1.5); j = nearest multiple of 1/256
// to m' - 0.75; r = m' G_j - 1 is exact (|r| < 2^-8); then
//   ln u = k ln 2 - ln G_j + r P(r),
//   P(r) = 1 - r/2 + r^2/3 - r^3/4 + r^4/5 - r^5/6 + r^6/7 - r^7/8
// (the Taylor series of ln(1 + r) / r, truncated below 2^-64), with the
// high-order part in 32-bit arithmetic, the rest in 64-bit, and the sum in
// 128-bit fixed point (scale 2^117) rounded once to binary64.
FP64I_HD double fp64i_log(double u, const uint64_t *tab)
{
    const uint64_t b = fp64i_bits(u);
    const uint32_t E = (uint32_t)(b >> 52);
    if (E - 1u >= 0x7FEu) return log(u);  // zero, subnormal, inf, nan, negative
    uint64_t M = (b & FP64I_FRAC) | FP64I_ONE;
    int k = (int)E - 1023;
    if (M >= (3ull << 51)) ++k;  // m' = m / 2 = M 2^-53
    else M <<= 1;                // m' = m = (2M) 2^-53
    const int j = (int)((M - (3ull << 51) + (1ull << 44)) >> 45);
    const uint32_t g = reinterpret_cast<const uint32_t *>(tab + 388)[j];
    const int64_t r = (int64_t)(M * (uint64_t)g - (1ull << 63));  // r 2^63, |r| < 2^55
    const uint64_t ra = r < 0 ? (uint64_t)(-r) : (uint64_t)r;
    // Q4 = 1/5 - r/6 + r^2/7 - r^3/8 at scale 2^33 (relative error 2^-31 suffices)
    const int64_t r32 = (int64_t)(int32_t)(r >> 25);  // r 2^38
    int32_t q = -(1 << 30);
    q = 1227133513 + (int32_t)(((int64_t)q * r32) >> 38);
    q = -1431655765 + (int32_t)(((int64_t)q * r32) >> 38);
    q = 1717986918 + (int32_t)(((int64_t)q * r32) >> 38);
    // r^2 2^78, Q2 = 1/3 - r/4 + r^2 Q4 at 2^64, P = 1 - r/2 + r^2 Q2 at 2^63
    const uint64_t R2 = fp64i_mulhi(ra << 8, ra << 8);
    const int64_t r2q4 = ((int64_t)(uint32_t)(R2 >> 30) * (int64_t)q) >> 17;
    const uint64_t Q2 = 0x5555555555555555ull - (uint64_t)(r >> 1) + (uint64_t)r2q4;
    const uint64_t P = (1ull << 63) - (uint64_t)(r >> 1) + (fp64i_mulhi(R2 << 1, Q2) >> 16);
    // B = r P at 2^117 (sign of r)
    const uint64_t pl = ra * P, ph = fp64i_mulhi(ra, P);
    const uint64_t blo = (pl >> 9) | (ph << 55), bhi = ph >> 9;
    // A = k ln 2 - ln G_j at 2^117
    const uint32_t ka = (uint32_t)(k < 0 ? -k : k);
    uint64_t lo = tab[387] * ka;
    uint64_t hi = tab[386] * ka + fp64i_mulhi(tab[387], ka);
    if (k < 0) {
        lo = ~lo + 1;
        hi = ~hi + (lo == 0);
    }
    {
        const uint64_t gl = tab[FP64I_LOG_N + j], gh = tab[j];
        const uint64_t nl = lo - gl;
        hi = hi - gh - (nl > lo);
        lo = nl;
    }
    if (r < 0) {
        const uint64_t nl = lo - blo;
        hi = hi - bhi - (nl > lo);
        lo = nl;
    } else {
        const uint64_t nl = lo + blo;
        hi = hi + bhi + (nl < lo);
        lo = nl;
    }
    // round the 128-bit value to binary64
    const uint64_t neg = hi >> 63;
    if (neg) {
        lo = ~lo + 1;
        hi = ~hi + (lo == 0);
    }
    if ((hi | lo) == 0) return 0.0;
    const int lz = hi ? fp64i_clz(hi) : 64 + fp64i_clz(lo);
    uint64_t h, l;
    if (lz >= 64) {
        h = lo << (lz - 64);
        l = 0;
    } else if (lz > 0) {
        h = (hi << lz) | (lo >> (64 - lz));
        l = lo << lz;
    } else {
        h = hi;
        l = lo;
    }
    uint64_t mant = h >> 11;
    mant += ((h >> 10) & 1u) & (uint64_t)((((h & 0x3FFu) | l) != 0) | (int)(mant & 1u));
    uint64_t ex = (uint64_t)(1023 + 10 - lz);
    if (mant >> 53) {
        mant >>= 1;
        ++ex;
    }
    return fp64i_from_bits((neg << 63) | (ex << 52) | (mant & FP64I_FRAC));
}

#if !defined(__CUDACC_RTC__)
// Host: the log table (layout above).  ln G_j = ln(g_j / 1024) and ln 2 from
// ln x = 2 atanh((x - 1)/(x + 1)), the series summed in 128-bit fixed point
// at 2^120 (error a few hundred units of 2^-120), then rounded to 2^117.

// (a b) 2^-120 for a, b < 2^121 (truncated; error below 3 units)
static inline unsigned __int128 fp64i_fx_mul(unsigned __int128 a, unsigned __int128 b)
{
    const uint64_t a1 = (uint64_t)(a >> 64), a0 = (uint64_t)a, b1 = (uint64_t)(b >> 64), b0 = (uint64_t)b;
    const unsigned __int128 p00 = (unsigned __int128)a0 * b0, p01 = (unsigned __int128)a0 * b1;
    const unsigned __int128 p10 = (unsigned __int128)a1 * b0, p11 = (unsigned __int128)a1 * b1;
    return (p11 << 8) + (p01 >> 56) + (p10 >> 56) + (p00 >> 120);
}

// 2 atanh(num / den) 2^120 for 0 <= num <= den / 3
static inline unsigned __int128 fp64i_atanh2_fx(uint64_t num, uint64_t den)
{
    const unsigned __int128 one = (unsigned __int128)1 << 120;
    const unsigned __int128 z = one / den * num + (one % den) * num / den;
    const unsigned __int128 z2 = fp64i_fx_mul(z, z);
    unsigned __int128 sum = 0, term = z;
    for (uint64_t i = 1; term != 0; i += 2) {
        sum += term / i;
        term = fp64i_fx_mul(term, z2);
    }
    return sum << 1;
}

// Returns 0, or -1 if a bucket's reduction would reach 2^-8 (it does not,
// for this choice of g_j; checked at both ends of every bucket).
static inline int fp64i_log_table(uint64_t *tab)
{
    for (int i = 0; i < FP64I_LOG_WORDS; ++i) tab[i] = 0;
    uint32_t *g = reinterpret_cast<uint32_t *>(tab + 388);
    auto store = [&](int hi_at, int lo_at, unsigned __int128 v120, bool negative) {
        unsigned __int128 v = (v120 + 4) >> 3;  // 2^120 -> 2^117, rounded
        if (negative) v = ~v + 1;
        tab[hi_at] = (uint64_t)(v >> 64);
        tab[lo_at] = (uint64_t)v;
    };
    store(386, 387, fp64i_atanh2_fx(1, 3), false);  // ln 2 = 2 atanh(1/3)
    for (int j = 0; j < FP64I_LOG_N; ++j) {
        const uint32_t gj = (uint32_t)((262144u + (192u + j) / 2) / (192u + j));
        g[j] = gj;
        // bucket j: M in [3 2^51 + j 2^45 - 2^44, 3 2^51 + j 2^45 + 2^44), clipped
        const uint64_t c = (3ull << 51) + ((uint64_t)j << 45);
        const uint64_t lo_m = j == 0 ? (3ull << 51) : c - (1ull << 44);
        const uint64_t hi_m = j == FP64I_LOG_N - 1 ? (3ull << 52) - 1 : c + (1ull << 44) - 1;
        const int64_t r_lo = (int64_t)(lo_m * (uint64_t)gj - (1ull << 63));
        const int64_t r_hi = (int64_t)(hi_m * (uint64_t)gj - (1ull << 63));
        const int64_t lim = (int64_t)1 << 55;
        if (r_lo <= -lim || r_lo >= lim || r_hi <= -lim || r_hi >= lim) return -1;
        const bool below = gj < 1024u;
        store(j, FP64I_LOG_N + j, fp64i_atanh2_fx(below ? 1024u - gj : gj - 1024u, gj + 1024u), below);
    }
    return 0;
}
#endif
