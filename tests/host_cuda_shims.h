// host_cuda_shims.h -- lets the library's device headers compile on the
// host for the tests: the CUDA qualifiers vanish, thread indices are those
// of a single lane, warp and block operations act on that lane alone, and
// each arithmetic intrinsic is the IEEE-754 operation it denotes (round to
// nearest; compile with -ffp-contract=off).
#pragma once
#include <math.h>
#include <stdint.h>
#include <string.h>

#define __device__
#define __global__
#define __constant__
#define __forceinline__ inline
#define __noinline__ __attribute__((noinline))
struct HostDim {
    unsigned x, y, z;
};
static HostDim threadIdx = {0, 0, 0}, blockIdx = {0, 0, 0}, blockDim = {32, 1, 1}, gridDim = {1, 1, 1};
struct uint4 {
    unsigned x, y, z, w;
};
static inline void __syncthreads() {}
static inline void __threadfence() {}
template <class T> static inline T __shfl_xor_sync(unsigned, T v, int, int = 32) { return v; }
template <class T> static inline T __shfl_sync(unsigned, T v, int, int = 32) { return v; }
template <class T> static inline T atomicAdd(T *p, T v) { const T o = *p; *p += v; return o; }
static inline double __dmul_rn(double a, double b) { return a * b; }
static inline double __dadd_rn(double a, double b) { return a + b; }
static inline double __dsub_rn(double a, double b) { return a - b; }
static inline double __ddiv_rn(double a, double b) { return a / b; }
static inline double __dsqrt_rn(double a) { return sqrt(a); }
static inline float __fmaf_rn(float a, float b, float c) { return fmaf(a, b, c); }
static inline long long __double_as_longlong(double d) { long long v; memcpy(&v, &d, 8); return v; }
static inline double __longlong_as_double(long long v) { double d; memcpy(&d, &v, 8); return d; }
static inline unsigned __float_as_uint(float f) { unsigned u; memcpy(&u, &f, 4); return u; }
static inline double __ull2double_rn(unsigned long long v) { return (double)v; }
static inline double __ll2double_rn(long long v) { return (double)v; }
static inline double __hiloint2double(int hi, int lo)
{
    return __longlong_as_double((long long)(((unsigned long long)(unsigned)hi << 32) | (unsigned)lo));
}

