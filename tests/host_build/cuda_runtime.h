// Stand-in for <cuda_runtime.h> in the host builds of the device headers (test harnesses only;
// the product is built with nvcc).  The CUDA qualifiers expand to nothing and each device
// intrinsic the headers use is written with host IEEE arithmetic: float and double operations
// rounded to nearest, std::fma for the fused multiply-add, bit copies through memcpy.  The
// approximations rsqrtf and rsqrt are 1/sqrt here (the device's are within 2 and 1 ulps).
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>

#define __host__
#define __device__
#define __forceinline__ inline
#define __noinline__

inline float __fadd_rn(float a, float b) { return a + b; }
inline float __fsub_rn(float a, float b) { return a - b; }
inline float __fmul_rn(float a, float b) { return a * b; }
inline float __fmaf_rn(float a, float b, float c) { return std::fma(a, b, c); }
inline float __frcp_rn(float a) { return 1.0f / a; }
inline float __fdividef(float a, float b) { return a / b; }
inline float rsqrtf(float a) { return 1.0f / std::sqrt(a); }
inline double rsqrt(double a) { return 1.0 / std::sqrt(a); }
inline float rsqrt(float a) { return 1.0f / std::sqrt(a); }

inline unsigned __float_as_uint(float f) { unsigned u; std::memcpy(&u, &f, 4); return u; }
inline float __uint_as_float(unsigned u) { float f; std::memcpy(&f, &u, 4); return f; }
inline long long __double_as_longlong(double d) { long long b; std::memcpy(&b, &d, 8); return b; }
inline double __longlong_as_double(long long b) { double d; std::memcpy(&d, &b, 8); return d; }
inline int __double2hiint(double d) { return (int)(unsigned)((unsigned long long)__double_as_longlong(d) >> 32); }
inline int __double2loint(double d) { return (int)(unsigned)((unsigned long long)__double_as_longlong(d) & 0xffffffffull); }
inline double __hiloint2double(int hi, int lo) {
  return __longlong_as_double((long long)(((unsigned long long)(unsigned)hi << 32) | (unsigned)lo));
}

// types the internal headers name in host declarations
typedef struct CUstream_st* cudaStream_t;
struct dim3 {
  unsigned x, y, z;
  dim3(unsigned a = 1, unsigned b = 1, unsigned c = 1) : x(a), y(b), z(c) {}
};

template <class T>
inline T __ldg(const T* p) { return *p; }
