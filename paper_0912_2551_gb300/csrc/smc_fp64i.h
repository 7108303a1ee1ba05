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

// The rare operands of the functions below go to the FP64 pipe through
// these out-of-line calls: kept out of line on the device so that the
// compiler cannot evaluate them speculatively next to the integer path.
#if defined(__CUDA_ARCH__)
#define FP64I_SLOW __device__ __noinline__
#else
#define FP64I_SLOW static
#endif
FP64I_SLOW double fp64i_slow_i2d(int64_t h) { return (double)h; }
FP64I_SLOW double fp64i_slow_div(double n, double d) { return n / d; }

// An integer h as a binary64, for 0 <= h < 2^53 built on the integer pipes
// (exact: leading bit found with clz, the significand shifted into place,
// the exponent added); negative h and h >= 2^53 (rare) take the conversion
// instruction, which rounds to nearest.  Same value as the conversion for
// every h.
FP64I_HD double fp64i_i2d(int64_t h)
{
    const uint64_t u = (uint64_t)h;
    if (__builtin_expect(u >> 53, 0)) return fp64i_slow_i2d(h);
    const int p = 63 - fp64i_clz(u | 1u);  // leading bit (h = 0 handled below)
    const uint64_t b = ((uint64_t)(1022 + p) << 52) + (u << (52 - p));
    return fp64i_from_bits(u ? b : 0ull);
}


// 1/delta for delta = md / 2^53 in [1/2, 1) (md in [2^52, 2^53)), as
// y = Y 2^-63 with Y <= 2^63 / delta < 2^64: a single-precision seed (relative
// error below 2^-21; 2 clamps to 2 - 2^-23), then two Newton steps
// y <- y (2 - delta y) in fixed point, the first with the seed as one 32-bit
// factor (error about 2^-42), the second in 64-bit (about 2^-62).
// Truncation keeps every step at or below 1/delta.
FP64I_HD uint64_t fp64i_recip63(uint64_t md)
{
    const uint64_t D = md << 11;  // delta 2^64
    const float s = fp64i_rcp_approx((float)(uint32_t)(D >> 40)) * 16777216.0f;
    uint32_t sb;
#if defined(__CUDA_ARCH__)
    sb = __float_as_uint(s);
#else
    memcpy(&sb, &s, 4);
#endif
    const uint32_t y24 = (sb >= 0x40000000u) ? 0xFFFFFFu : ((sb & 0x7FFFFFu) | 0x800000u);
    uint64_t Y;
    {
        // Y0 = y24 2^40: W = (2^88 - D y24) 2^-24, Y = y24 W 2^-23
        const uint64_t pl = (uint64_t)(uint32_t)D * y24;
        const uint64_t pm = (D >> 32) * (uint64_t)y24 + (pl >> 32);  // D y24 = pm 2^32 + low word of pl
        const uint32_t low = (uint32_t)pl;
        const uint64_t nm = (1ull << 56) - pm - (low != 0u);          // 2^88 - D y24 = nm 2^32 + nl
        const uint32_t nl = 0u - low;
        const uint64_t W = (nm << 8) | (nl >> 24);
        const uint64_t ql = (uint64_t)(uint32_t)W * y24;
        const uint64_t qm = (W >> 32) * (uint64_t)y24 + (ql >> 32);  // y24 W = qm 2^32 + low word of ql
        Y = (qm << 9) | ((ql & 0xFFFFFFFFull) >> 23);
    }
    {
        // W = high word of 2^128 - D Y, Y = Y W 2^-63
        const uint64_t pl = D * Y, ph = fp64i_mulhi(D, Y);
        const uint64_t W = ~ph + (pl == 0);
        const uint64_t ql = Y * W, qh = fp64i_mulhi(Y, W);
        Y = (qh << 1) | (ql >> 63);
    }
    return Y;
}

// n / d, correctly rounded (nearest, ties to even).  The integer path has
// no branch (so the compiler can interleave it with independent work); the
// operands and quotients it does not cover are redone by the FP64 division
// at the end.
FP64I_HD double fp64i_div(double n, double d)
{
    const uint64_t bn = fp64i_bits(n), bd = fp64i_bits(d);
    const uint32_t en = (uint32_t)(bn >> 52), ed = (uint32_t)(bd >> 52);  // sign bit included
    // zero, subnormal, inf, nan or negative operands
    bool special = (en - 1u >= 0x7FEu) | (ed - 1u >= 0x7FEu);
    uint64_t mn = (bn & FP64I_FRAC) | FP64I_ONE;
    const uint64_t md = (bd & FP64I_FRAC) | FP64I_ONE;
    const bool lt = mn < md;
    mn <<= lt;                                       // mn / md in [1, 2)
    int e = (int)en - (int)ed + 1023 - (int)lt;      // biased exponent of the quotient
    const uint64_t Y = fp64i_recip63(md);
    // Qt = floor(mn 2^53 / md), in [2^53, 2^54): the estimate mn Y 2^-63 is
    // Qt or Qt - 1 (Y <= 2^63 / delta, relative error about 2^-62); the
    // exact remainder (64-bit wrap-around arithmetic) settles it
    uint64_t qt = (fp64i_mulhi(mn, Y) << 1) | ((mn * Y) >> 63);
    uint64_t rem = (mn << 53) - qt * md;
    for (int c = 0; c < 2; ++c) {
        const bool up = rem >= md;
        qt += up;
        rem -= up ? md : 0ull;
    }
    uint64_t q = qt >> 1;
    q += (qt & 1u) & (uint64_t)((rem != 0) | (int)(q & 1u));
    const uint64_t carry = q >> 53;  // rounded up to 2: next binade
    q >>= carry;
    e += (int)carry;
    special |= (e < 1) | (e > 2046);  // subnormal or infinite quotient
    if (__builtin_expect(special, 0)) return fp64i_slow_div(n, d);
    return fp64i_from_bits(((uint64_t)e << 52) | (q & FP64I_FRAC));
}

// |r| P(r) at scale 2^117 as (lo, hi), for r = m' G_j - 1 given as r 2^63
// (|r| < 2^-8): P(r) = 1 - r/2 + r^2/3 - r^3/4 + r^4/5 - r^5/6 + r^6/7 - r^7/8,
// the Taylor series of ln(1 + r) / r truncated below 2^-64, with the terms
// from r^4 on in 32-bit arithmetic (relative error 2^-31 suffices there) and
// the rest in 64-bit fixed point (relative error of the result about 2^-63).
FP64I_HD void fp64i_log1p_abs(int64_t r, uint64_t &blo, uint64_t &bhi)
{
    const uint64_t ra = r < 0 ? (uint64_t)(-r) : (uint64_t)r;
    // Q4 = 1/5 - r/6 + r^2/7 - r^3/8 at scale 2^33
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
    const uint64_t pl = ra * P, ph = fp64i_mulhi(ra, P);
    blo = (pl >> 9) | (ph << 55);
    bhi = ph >> 9;
}

// A positive 128-bit value v (scale 2^117) rounded to binary64, nearest-even.
FP64I_HD uint64_t fp64i_round117(uint64_t lo, uint64_t hi)
{
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
    uint64_t ex = (uint64_t)(1023 + 10 - lz);  // leading bit 127 - lz at scale 2^117
    if (mant >> 53) {
        mant >>= 1;
        ++ex;
    }
    return (ex << 52) | (mant & FP64I_FRAC);
}

// The same for 2^64 <= v < 2^127 (the leading bit in the high word, below
// its top bit): no branch.
FP64I_HD uint64_t fp64i_round117_hi(uint64_t lo, uint64_t hi)
{
    const int lz = fp64i_clz(hi);  // 1..63
    const uint64_t h = (hi << lz) | (lo >> (64 - lz)), l = lo << lz;
    uint64_t mant = h >> 11;
    mant += ((h >> 10) & 1u) & (uint64_t)((((h & 0x3FFu) | l) != 0) | (int)(mant & 1u));
    const uint64_t carry = mant >> 53;
    return ((uint64_t)(1023 + 10 - lz + (int)carry) << 52) + ((mant >> carry) & FP64I_FRAC);
}

// The reduction of m' = M 2^-53 (M in [3 2^51, 3 2^52)): bucket j and
// r = m' G_j - 1 as r 2^63 (exact, |r| < 2^55).
FP64I_HD int64_t fp64i_reduce(uint64_t M, const uint64_t *tab, int &j)
{
    j = (int)((M - (3ull << 51) + (1ull << 44)) >> 45);
    const uint32_t g = reinterpret_cast<const uint32_t *>(tab + 388)[j];
    return (int64_t)(M * (uint64_t)g - (1ull << 63));
}

// ln u.  u = 2^k m' with m' in [0.75, 1.5); j = nearest multiple of 1/256
// to m' - 0.75; r = m' G_j - 1 is exact (|r| < 2^-8); then
//   ln u = k ln 2 - ln G_j + r P(r)
// summed in 128-bit fixed point (scale 2^117) and rounded once to binary64.
FP64I_HD double fp64i_log(double u, const uint64_t *tab)
{
    const uint64_t b = fp64i_bits(u);
    const uint32_t E = (uint32_t)(b >> 52);
    if (E - 1u >= 0x7FEu) return log(u);  // zero, subnormal, inf, nan, negative
    uint64_t M = (b & FP64I_FRAC) | FP64I_ONE;
    int k = (int)E - 1023;
    if (M >= (3ull << 51)) ++k;  // m' = m / 2 = M 2^-53
    else M <<= 1;                // m' = m = (2M) 2^-53
    int j;
    const int64_t r = fp64i_reduce(M, tab, j);
    uint64_t blo, bhi;
    fp64i_log1p_abs(r, blo, bhi);
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
    const uint64_t neg = hi >> 63;
    if (neg) {
        lo = ~lo + 1;
        hi = ~hi + (lo == 0);
    }
    if ((hi | lo) == 0) return 0.0;
    return fp64i_from_bits((neg << 63) | fp64i_round117(lo, hi));
}

// -ln(n 2^-53) for an odd integer 1 <= n < 2^53: the SSA's uniform
// u = (2v + 1) 2^-53 taken as its integer n, so neither u nor its bit
// pattern is formed; the same arithmetic as -fp64i_log(u) (equal bits):
//   -ln u = |k| ln 2 + ln G_j - r P(r),  k <= 0, the sum positive.
FP64I_HD void fp64i_neglog53_fx(uint64_t n, const uint64_t *tab, uint64_t &lo, uint64_t &hi)
{
    const int p = 63 - fp64i_clz(n);  // u = (n 2^-p) 2^(p - 53), n 2^-p in [1, 2)
    uint64_t M = n << (52 - p);       // m 2^52
    int ka = 53 - p;                  // -k
    if (M >= (3ull << 51)) --ka;      // m' = m / 2 = M 2^-53
    else M <<= 1;                     // m' = m = (2M) 2^-53
    int j;
    const int64_t r = fp64i_reduce(M, tab, j);
    uint64_t blo, bhi;
    fp64i_log1p_abs(r, blo, bhi);
    lo = tab[387] * (uint32_t)ka;
    hi = tab[386] * (uint32_t)ka + fp64i_mulhi(tab[387], (uint32_t)ka);
    {
        const uint64_t gl = tab[FP64I_LOG_N + j], gh = tab[j];
        const uint64_t nl = lo + gl;
        hi = hi + gh + (nl < lo);
        lo = nl;
    }
    if (r < 0) {
        const uint64_t nl = lo + blo;
        hi = hi + bhi + (nl < lo);
        lo = nl;
    } else {
        const uint64_t nl = lo - blo;
        hi = hi - bhi - (nl > lo);
        lo = nl;
    }
}

FP64I_HD double fp64i_neglog53(uint64_t n, const uint64_t *tab)
{
    uint64_t lo, hi;
    fp64i_neglog53_fx(n, tab, lo, hi);
    return fp64i_from_bits(fp64i_round117_hi(lo, hi));  // the sum is in [2^64, 2^123)
}

// -ln(n 2^-53) normalised from the 128-bit sum above: S = sm 2^(-53 - lz),
// sm in [2^63, 2^64), the sum's top 64 bits (truncated: relative error
// below 2^-63).  The SSA draws it one event ahead of its use.
FP64I_HD void fp64i_neglog53_norm(uint64_t n, const uint64_t *tab, uint64_t &sm, int &lz)
{
    uint64_t lo, hi;
    fp64i_neglog53_fx(n, tab, lo, hi);
    lz = fp64i_clz(hi);  // hi >= 1: the sum is at least 2^64
    sm = (hi << lz) | ((lo >> 1) >> (63 - lz));
}

// tau = S / a for S = sm 2^(-53 - lz) from fp64i_neglog53_norm and a > 0
// (Eq. 2a), rounded once: S times the reciprocal of a (fp64i_recip63), the
// high word of the 64 x 64-bit product rounded to 53 bits.  Each factor and
// the product are truncated, so the unrounded value lies below S / a by a
// relative 2^-60 at most, and the result is within 0.5 + 2^-7 ulp of S / a
// (faithful; correctly rounded but within 2^-7 ulp of a rounding midpoint).
// S / a is never a midpoint (S is a logarithm of a rational other than 1),
// so a computed value exactly at one rounds up.  Zero, subnormal, infinite,
// negative or NaN a, and quotients outside the normal range, take the
// division of the rounded logarithm by a (within one ulp).
FP64I_HD double fp64i_tau(uint64_t sm, int lz, double a)
{
    const uint64_t ba = fp64i_bits(a);
    const uint32_t ea = (uint32_t)(ba >> 52);  // sign bit included
    const uint64_t Y = fp64i_recip63((ba & FP64I_FRAC) | FP64I_ONE);
    // S / a = sm Y 2^(906 - lz - ea); PH = floor(sm Y 2^-64) in [2^62, 2^64)
    const uint64_t ph = fp64i_mulhi(sm, Y);
    const uint32_t top = (uint32_t)(ph >> 63);
    uint64_t m = ph >> (10 + top);
    m += (ph >> (9 + top)) & 1u;          // guard bit: round half up (no exact midpoint)
    const uint64_t carry = m >> 53;
    m >>= carry;
    const int e = 2055 + (int)top + (int)carry - lz - (int)ea;
    if (__builtin_expect((ea - 1u >= 0x7FEu) | (e < 1) | (e > 2046), 0)) {
        uint64_t s53 = (sm >> 11) + ((sm >> 10) & 1u);  // the logarithm rounded to 53 bits
        const uint64_t c2 = s53 >> 53;
        s53 >>= c2;
        return fp64i_slow_div(fp64i_from_bits(((uint64_t)(1023 + 10 - lz + (int)c2) << 52) + (s53 & FP64I_FRAC)), a);
    }
    return fp64i_from_bits(((uint64_t)e << 52) + (m & FP64I_FRAC));
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
