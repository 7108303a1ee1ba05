// Fixed-width integer types for the run-time compiled kernels (NVRTC
// provides no C library headers); the sizes match the LP64 host ABI.
#pragma once
typedef signed char int8_t;
typedef short int16_t;
typedef int int32_t;
typedef long long int64_t;
typedef unsigned char uint8_t;
typedef unsigned short uint16_t;
typedef unsigned int uint32_t;
typedef unsigned long long uint64_t;
