// Host check of the integer-pipe binary64 division and logarithm
// (paper_0912_2551_gb300/csrc/smc_fp64i.h) against the platform's
// arithmetic: the division bit for bit against IEEE-754 division, the
// logarithm against long double logl in ulps.  Prints one line of
// key=value pairs; exit status 0 when every check holds.
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "smc_fp64i.h"

static uint64_t s_state = 0x9E3779B97F4A7C15ull;
static uint64_t next_u64()  // splitmix64
{
    uint64_t z = (s_state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double bits_to_double(uint64_t b)
{
    double x;
    memcpy(&x, &b, 8);
    return x;
}

static uint64_t double_bits(double x)
{
    uint64_t b;
    memcpy(&b, &x, 8);
    return b;
}

static double ulp_error(double got, double u)
{
    const long double ref = logl((long double)u);
    const double rd = (double)ref;
    double ulp = rd == 0.0 ? 4.9e-324 : fabs(nextafter(rd, INFINITY) - rd);
    if (fabs(nextafter(rd, 0.0) - rd) < ulp && fabs(ref) < fabs((long double)rd)) ulp = fabs(nextafter(rd, 0.0) - rd);
    return (double)(fabsl((long double)got - ref) / (long double)ulp);
}

int main(int argc, char **argv)
{
    long n = argc > 1 ? atol(argv[1]) : 2000000;
    static uint64_t tab[FP64I_LOG_WORDS];
    if (fp64i_log_table(tab)) {
        printf("table=fail\n");
        return 1;
    }
    // division: random positive normals over the full exponent range, then
    // significands near the rounding boundaries, then special operands
    long div_bad = 0, div_n = 0;
    for (long i = 0; i < n; ++i) {
        double a, b;
        const int kind = (int)(i % 4);
        if (kind == 0) {  // uniform bit patterns (any class)
            a = bits_to_double(next_u64());
            b = bits_to_double(next_u64());
        } else if (kind == 1) {  // moderate exponents, both positive
            a = bits_to_double((next_u64() & 0x000FFFFFFFFFFFFFull) | ((uint64_t)(1023 - 60 + next_u64() % 120) << 52));
            b = bits_to_double((next_u64() & 0x000FFFFFFFFFFFFFull) | ((uint64_t)(1023 - 60 + next_u64() % 120) << 52));
        } else if (kind == 2) {  // exact quotients and their neighbours
            const double q = bits_to_double((next_u64() & 0x000FFFFFFFFFFFFFull) | (1023ull << 52));
            b = bits_to_double((next_u64() & 0x000FFFFFFFFFFFFFull) | (1023ull << 52));
            a = q * b;
            a = bits_to_double(double_bits(a) + (int)(next_u64() % 5) - 2);
        } else if (kind == 3 && (i & 4)) {  // divisors just above and below powers of two
            a = bits_to_double((next_u64() & 0x000FFFFFFFFFFFFFull) | ((uint64_t)(1000 + next_u64() % 48) << 52));
            const uint64_t f = (i & 8) ? (next_u64() >> 34) : (0x000FFFFFFFFFFFFFull - (next_u64() >> 34));
            b = bits_to_double(f | ((uint64_t)(1000 + next_u64() % 48) << 52));
        } else {  // few significand bits (ties and short patterns)
            a = bits_to_double((next_u64() & 0x000FF00000000000ull) | ((uint64_t)(1000 + next_u64() % 48) << 52));
            b = bits_to_double((next_u64() & 0x000F000000000000ull) | ((uint64_t)(1000 + next_u64() % 48) << 52));
        }
        const double got = fp64i_div(a, b), want = a / b;
        ++div_n;
        if (double_bits(got) != double_bits(want) && !(got != got && want != want)) {
            if (div_bad < 5) printf("div_mismatch a=%a b=%a got=%a want=%a\n", a, b, got, want);
            ++div_bad;
        }
    }
    const double edges[][2] = {{1.0, 3.0}, {2.0, 3.0}, {1.0, 1.0}, {3.0, 2.0}, {1e308, 1e-10}, {1e-300, 1e10},
                               {2.2250738585072014e-308, 2.0}, {4.0, 2.0}, {1.0, 0.0}, {0.0, 1.0}, {-1.0, 3.0},
                               {1.9999999999999998, 1.0000000000000002}, {1.0000000000000002, 1.9999999999999998}};
    for (const auto &e : edges) {
        const double got = fp64i_div(e[0], e[1]), want = e[0] / e[1];
        ++div_n;
        if (double_bits(got) != double_bits(want)) {
            printf("div_mismatch a=%a b=%a got=%a want=%a\n", e[0], e[1], got, want);
            ++div_bad;
        }
    }
    // logarithm: the SSA uniforms (2v + 1) 2^-53, values near 1, bucket
    // edges and general positive doubles
    double worst = 0.0, worst_u = 0.0;
    long log_n = 0, rounded_ok = 0;
    auto check = [&](double u) {
        const double got = fp64i_log(u, tab);
        const double err = ulp_error(got, u);
        ++log_n;
        rounded_ok += err <= 0.5;
        if (err > worst) {
            worst = err;
            worst_u = u;
        }
    };
    for (long i = 0; i < n; ++i) {
        const uint64_t v = next_u64() >> 12;
        check(((double)(2 * v + 1)) * 0x1p-53);
    }
    for (long i = 0; i < n / 4; ++i) {
        const uint64_t v = next_u64() >> 12;
        const double d = ((double)(2 * v + 1)) * 0x1p-59;
        check(1.0 - d);
        check(1.0 + d);
    }
    for (int j = 0; j < FP64I_LOG_N; ++j)
        for (int s = -2; s <= 2; ++s) {
            const double c = 0.75 + (j + 0.5) / 256.0;
            check(bits_to_double(double_bits(c) + s));
        }
    for (long i = 0; i < n / 4; ++i) check(exp(-700.0 + 1400.0 * (double)(next_u64() >> 11) * 0x1p-53));
    // the SSA form: -ln((2v + 1) 2^-53) from the integer, equal bits to -ln u
    long neglog_bad = 0;
    for (long i = 0; i < n; ++i) {
        const uint64_t v = (i < 64) ? (uint64_t)i : (i < 128 ? (1ull << 52) - 1 - (uint64_t)(i - 64) : next_u64() >> 12);
        const uint64_t nn = 2 * v + 1;
        const double u = (double)nn * 0x1p-53;
        const double want = -fp64i_log(u, tab), got = fp64i_neglog53(nn, tab);
        if (double_bits(got) != double_bits(want)) {
            if (neglog_bad < 5) printf("neglog53_mismatch n=%llu got=%a want=%a\n", (unsigned long long)nn, got, want);
            ++neglog_bad;
        }
    }
    const double log_edges[] = {0x1p-53, 1 - 0x1p-53, 0.5, 0.75, 1.0, 1.5, 2.0, 3.0, 0.1, 1e-300, 1e300,
                                1.7976931348623157e308, 2.2250738585072014e-308};
    for (double u : log_edges) check(u);
    // the exact conversion of integers (counts, propensity products), bit for
    // bit against the IEEE conversion
    long conv_bad = 0;
    for (long i = 0; i < n; ++i) {
        uint64_t h;
        switch (i % 4) {
        case 0: h = next_u64() >> (next_u64() % 64); break;
        case 1: h = (uint64_t)(i / 4); break;
        case 2: h = (1ull << (i / 4 % 64)) + (uint64_t)((int)(next_u64() % 5) - 2); break;
        default: h = ((1ull << 53) - 3 + (uint64_t)(i / 4 % 7)) << (i / 28 % 4); break;
        }
        const int64_t hs = (i % 8 == 7) ? -(int64_t)(h >> 1) : (int64_t)h;  // negative values too
        if (double_bits(fp64i_i2d(hs)) != double_bits((double)hs)) {
            if (conv_bad < 5) printf("i2d_mismatch h=%lld\n", (long long)hs);
            ++conv_bad;
        }
    }
    // tau = -ln(n 2^-53) / a rounded once (fp64i_neglog53_norm + fp64i_tau)
    // against the long-double quotient, in ulps of the result
    double tau_worst = 0.0;
    long tau_n = 0, tau_cr = 0, tau_bad = 0;
    for (long i = 0; i < n; ++i) {
        const uint64_t nn = (i % 7 == 0) ? ((1ull << 53) - 1 - 2 * (next_u64() % 4096))      // u near 1
                            : (i % 7 == 1) ? (((next_u64() >> (12 + next_u64() % 52)) << 1) | 1u)  // small u
                                           : ((next_u64() >> 11) | 1u);
        double a;
        if (i % 3 == 0) a = bits_to_double((next_u64() & 0x000FFFFFFFFFFFFFull) | ((uint64_t)(1023 - 30 + next_u64() % 60) << 52));
        else if (i % 3 == 1) a = (double)(1 + (next_u64() >> (next_u64() % 64)));  // integer-valued sums
        else a = bits_to_double((next_u64() & 0x000FFFFFFFFFFFFFull) | ((uint64_t)(1 + next_u64() % 2046) << 52));
        uint64_t sm;
        int lz;
        fp64i_neglog53_norm(nn, tab, sm, lz);
        const double got = fp64i_tau(sm, lz, a);
        const long double ref = -logl((long double)nn * 0x1p-53L) / (long double)a;
        const double rd = (double)ref;
        if (!(rd > 0.0) || rd == INFINITY || rd < 2.2250738585072014e-308) {  // outside the normal range
            tau_bad += got != rd && !(got == 0.0 && rd == 0.0) && fabsl((long double)got - ref) > 1e-300L;
            continue;
        }
        double ulp = nextafter(rd, INFINITY) - rd;
        const double dn = rd - nextafter(rd, 0.0);
        if (dn < ulp && (long double)rd > ref) ulp = dn;
        const double err = (double)(fabsl((long double)got - ref) / (long double)ulp);
        ++tau_n;
        tau_cr += err <= 0.5;
        if (err > tau_worst) tau_worst = err;
    }
    {
        uint64_t sm;
        int lz;
        fp64i_neglog53_norm(12345u, tab, sm, lz);
        const double l = fp64i_neglog53(12345u, tab);
        tau_bad += fp64i_tau(sm, lz, 0.0) != INFINITY;                    // absorbing: a_0 = 0
        tau_bad += fp64i_tau(sm, lz, 1.0) != l;                           // the logarithm itself
        tau_bad += fp64i_tau(sm, lz, 4.9e-324) != l / 4.9e-324;           // subnormal a (overflow)
        tau_bad += fp64i_tau(sm, lz, 1e-310) != l / 1e-310;
    }
    const double special = fp64i_log(0.0, tab);
    const bool special_ok = special == -INFINITY && fp64i_log(-1.0, tab) != fp64i_log(-1.0, tab) &&
                            fp64i_log(1.0, tab) == 0.0;
    const double frac_ok = (double)rounded_ok / (double)log_n;
    printf("div_checked=%ld div_mismatches=%ld log_checked=%ld log_max_ulp=%.6f log_max_at=%a "
           "log_correctly_rounded=%.7f special_ok=%d neglog53_mismatches=%ld i2d_mismatches=%ld "
           "tau_checked=%ld tau_max_ulp=%.6f tau_correctly_rounded=%.7f tau_bad=%ld\n",
           div_n, div_bad, log_n, worst, worst_u, frac_ok, (int)special_ok, neglog_bad, conv_bad, tau_n,
           tau_worst, (double)tau_cr / (double)tau_n, tau_bad);
    return (div_bad == 0 && worst <= 0.502 && frac_ok >= 0.9995 && special_ok && neglog_bad == 0 && conv_bad == 0 &&
            tau_worst <= 0.51 && tau_bad == 0)
               ? 0
               : 1;
}
