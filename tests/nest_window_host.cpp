// Host check of the trace monitor's window bounds (smc_nest.h:
// nest_last_within, nest_first_reaching): for window offsets t_j and
// bounds a, b of every kind (zero, small decimals, random, subnormal, near
// the top of the double range, +inf), the integer tests bits(t) <= last and
// bits(t) >= first must agree with the rounded subtractions t - t_j <= b and
// t - t_j >= a for every time t in a few-ulp neighbourhood of the boundary,
// of t_j + b, and for random times.  A bound that comes back -1 (the scan
// then subtracts) is counted; it must not happen for ordinary values.
// Output: "cases checks mismatches fallbacks_ordinary fallbacks_extreme".
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <random>
#include <vector>

#include "smc_nest.h"

static int64_t bits(double x) { return nest_bits(x); }
static double from(int64_t b) { return nest_from_bits(b); }

int main()
{
    std::mt19937_64 rng(20260412);
    std::uniform_real_distribution<double> U(0.0, 1.0);
    std::vector<double> offsets = {0.0, 0.25, 0.5, 1.0, 3.0, 19.75, 20.0, 100.0, 1e-310, 1e300, 1.7e308};
    std::vector<double> bounds = {0.0, 0.5, 1.0, 2.0, 3.0, 20.0, 0.1, 1e-320, 1e-300, 1e300, 1.7e308, INFINITY};
    for (int k = 0; k < 400; ++k) {
        offsets.push_back(100.0 * U(rng));
        offsets.push_back(ldexp(U(rng), (int)(U(rng) * 60) - 30));
        bounds.push_back(10.0 * U(rng));
        bounds.push_back(ldexp(U(rng), (int)(U(rng) * 60) - 30));
    }
    long long cases = 0, checks = 0, bad = 0, fb_ord = 0, fb_ext = 0;
    const int64_t inf = bits(INFINITY);
    for (double tj : offsets)
        for (double b : bounds) {
            ++cases;
            const bool extreme = tj > 1e299 || (b > 1e299 && b < INFINITY);
            const int64_t last = nest_last_within(tj, b);
            const int64_t first = nest_first_reaching(tj, b);
            if (last < 0 || (first < 0 && b < INFINITY)) {
                if (extreme) ++fb_ext; else ++fb_ord;
            }
            std::vector<int64_t> xs;
            const int64_t centres[] = {bits(tj), bits(tj + b), last, first};
            for (int64_t c : centres) {
                if (c < 0) continue;
                for (int64_t d = -8; d <= 8; ++d) {
                    const int64_t x = c + d;
                    if (x >= 0 && x <= inf) xs.push_back(x);
                }
            }
            for (int r = 0; r < 16; ++r) xs.push_back(bits(tj + (b < 1e300 ? 2.0 * b + 1.0 : 1e300) * U(rng)));
            for (int64_t x : xs) {
                const double t = from(x);
                if (t < tj) continue;  // the scans look at times t >= t_j only
                ++checks;
                if (last >= 0 && ((x <= last) != (t - tj <= b))) {
                    if (bad < 10) printf("last: tj %a b %a t %a\n", tj, b, t);
                    ++bad;
                }
                if (b < INFINITY && first >= 0 && ((x >= first) != (t - tj >= b))) {
                    if (bad < 10) printf("first: tj %a a %a t %a\n", tj, b, t);
                    ++bad;
                }
            }
        }
    printf("%lld %lld %lld %lld %lld\n", cases, checks, bad, fb_ord, fb_ext);
    return bad ? 1 : 0;
}
