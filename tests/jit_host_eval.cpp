// Evaluates a generated model header (jit_model.h, from
// tests/jit_header_dump.cpp) on the host: the CUDA intrinsics it calls are
// replaced by the IEEE-754 operations they denote (round to nearest, no
// contraction: compile with -ffp-contract=off), and its integer-to-double
// conversions are the library's own (smc_fp64i.h), so the FP64 results are
// those of the GPU bit for bit.  Reads R rate constants, then states (S
// counts each) until end of input; per state prints the FP64 prefix sums
// (bit patterns, hex), the positive-propensity mask, the FP32 prefix sums,
// the atom bits, and for each reaction the state after x += v_j.
#include <inttypes.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#define __device__
#define __forceinline__ inline
static inline double __dmul_rn(double a, double b) { return a * b; }
static inline double __dadd_rn(double a, double b) { return a + b; }
static inline double __ddiv_rn(double a, double b) { return a / b; }
static inline float __fmul_rn(float a, float b) { return a * b; }
static inline float __fadd_rn(float a, float b) { return a + b; }
static inline float __fdiv_rn(float a, float b) { return a / b; }
static inline float __fmaf_rn(float a, float b, float c) { return fmaf(a, b, c); }
static inline double __fma_rn(double a, double b, double c) { return fma(a, b, c); }
static inline long long __double_as_longlong(double d)
{
    long long v;
    memcpy(&v, &d, 8);
    return v;
}
// the integer-pipe conversions the generated code calls (smc_fp64i.h,
// compiled for the host): their exactness is part of what is checked
#include "smc_fp64i.h"
static inline double int_to_double(long long v) { return fp64i_i2d(v); }

#include "jit_model.h"

int main()
{
    double c[JR];
    float cf[JR];
    for (int k = 0; k < JR; ++k) {
        if (scanf("%lf", &c[k]) != 1) return 2;
        cf[k] = (float)c[k];
    }
    int32_t x[JS];
    for (;;) {
        for (int i = 0; i < JS; ++i)
            if (scanf("%d", &x[i]) != 1) return 0;
        double pre[JR];
        float pref[JR];
        uint32_t pos = 0, posf = 0;
        jit_props_plain(x, c, pre, pos);
        jit_props_mixed(x, cf, pref, posf);
        printf("P");
        for (int k = 0; k < JR; ++k) {
            uint64_t b;
            memcpy(&b, &pre[k], 8);
            printf(" %016" PRIx64, b);
        }
        printf("\nM %u %u", pos, posf);
        for (int k = 0; k < JR; ++k) printf(" %.9g", (double)pref[k]);
#if JNA > 0
        printf("\nA %u", jit_atoms(x));
#else
        printf("\nA 0");
#endif
        for (int j = 0; j < JR; ++j) {
            int32_t y[JS];
            memcpy(y, x, sizeof(y));
#ifdef JIT_MEDIUM
            jit_apply_row(kJitDelta + j * JW, y, 1);
#else
            jit_apply(j, y, 1);
#endif
            printf("\nX");
            for (int i = 0; i < JS; ++i) printf(" %d", y[i]);
        }
        printf("\n");
    }
}
