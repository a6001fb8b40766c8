// hzn_f32x2.cuh -- double-word ("float-float") arithmetic for the FP32 pipes.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2: about 48
// significant bits, relative rounding error of order u^2 = 2^-48 per operation (FP64: 2^-53).
// On a GPU whose FP64 pipe issues 2 operations per clock per SM and whose FP32 pipes issue 128,
// a double-word operation of 6-12 FP32 instructions costs a fraction of one FP64 operation.
//
// The operations are built from three error-free transformations:
//   TwoSum(a, b)   s + e = a + b exactly, any a, b        (Knuth, TAOCP vol. 2, §4.2.2)
//   Fast2Sum(a, b) s + e = a + b exactly, |a| >= |b|      (Dekker, Numer. Math. 18, 1971)
//   TwoProd(a, b)  p + e = a * b exactly, with one FMA
// and follow the algorithms and error bounds of Joldes, Muller and Popescu, "Tight and rigorous
// error bounds for basic building blocks of double-word arithmetic", ACM TOMS 44(2), 2017:
// the sum is their "sloppy" double-word addition (absolute error of order u^2 (|x| + |y|),
// the same kind of bound a rounded FP64 input carries into a cancellation), the product their
// FMA-based double-word multiplication (relative error <= 5u^2); quotient, square root and
// inverse square root are one Newton correction of an FP32 approximation with the residual
// formed exactly (relative error of order u^2).
//
// Range: the exponent range is FP32's.  Values below about 1e-31 keep fewer than 48 bits (lo
// becomes subnormal); values below 1.2e-38 are flushed to 0 by split().
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace hzn {
// A namespace of its own, so that sqrt, fabs, fmin, ... of f32x2 are found only by
// argument-dependent lookup and never hide the double and float functions.
namespace dw {

struct f32x2 {
  float hi, lo;

  f32x2() = default;
  __host__ __device__ constexpr f32x2(float h, float l) : hi(h), lo(l) {}
  // From a double: hi = round(x), lo = round(x - hi) (x - hi is exact in double).  Meant for
  // constants, which the compiler folds; run-time values go through split().
  __host__ __device__ f32x2(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ explicit f32x2(float x) : hi(x), lo(0.0f) {}
  __host__ __device__ explicit f32x2(int x) : hi((float)x), lo(0.0f) {}
};

// ---- error-free transformations
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// ---- conversions by integer operations (FP32<->FP64 conversion instructions issue at the FP64
// pipe's rate on this GPU; these use the integer and FP32 pipes only)

// double -> pair: hi = x with its mantissa truncated to 24 bits (exact bit copy), lo = the
// remaining 29 mantissa bits as a float, then renormalised.  |x| below 2^-126 gives 0; |x| must
// be below 2^128 (the FP32 range).
__device__ __forceinline__ f32x2 split(double x) {
  const unsigned hw = (unsigned)__double2hiint(x), lw = (unsigned)__double2loint(x);
  const unsigned sign = hw & 0x80000000u;
  const int E = (int)((hw >> 20) & 0x7ffu);  // biased FP64 exponent
  const int e = E - 1023;
  const unsigned mh = ((hw & 0xfffffu) << 3) | (lw >> 29);
  const float h = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | mh);
  // remainder rem < 2^29, worth rem 2^(e-52): rem = a 2^6 + b with a < 2^23, b < 2^6, each
  // made exact in FP32 by the 2^23 offset trick, then scaled by 2^(e-52) (as 2^(e+12) 2^-64
  // when 2^(e-52) is below the FP32 normal range)
  const unsigned rem = lw & 0x1fffffffu;
  const float fa = __fsub_rn(__uint_as_float(0x4b000000u | (rem >> 6)), 8388608.0f);
  const float fb = __fsub_rn(__uint_as_float(0x4b000000u | (rem & 63u)), 8388608.0f);
  const float r = __fmaf_rn(fa, 64.0f, fb);
  const bool low = e < -74;
  const float sc = __uint_as_float((unsigned)(e - 52 + (low ? 64 : 0) + 127) << 23);
  float l = __fmul_rn(__fmul_rn(r, sc), low ? 5.421010862427522e-20f : 1.0f);  // 2^-64
  l = __uint_as_float(__float_as_uint(l) | sign);
  float zh, zl;
  zh = __fadd_rn(h, l);
  zl = __fsub_rn(l, __fsub_rn(zh, h));
  const bool tiny = e < -126;
  return f32x2(tiny ? 0.0f : zh, tiny ? 0.0f : zl);
}

// float -> double by bit copy (exact for normal floats; 0 for zero and subnormals).
__device__ __forceinline__ double widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned E = (u >> 23) & 0xffu;
  const unsigned hw = (u & 0x80000000u) | ((E + 896u) << 20) | ((u & 0x7fffffu) >> 3);
  const unsigned lw = u << 29;
  return E == 0u ? 0.0 : __hiloint2double((int)hw, (int)lw);
}

// float -> double, exact, by integer operations for finite floats (zero for subnormals, which
// lie below 1.2e-38); infinities and NaNs take the conversion instruction, so they propagate.
__device__ __forceinline__ double widen_exact(float f) {
  if (((__float_as_uint(f) >> 23) & 0xffu) == 0xffu) return (double)f;
  return widen(f);
}

// double -> float rounded to nearest (ties to even) by integer operations, for results in the
// FP32 normal range and for zeros (FP64 subnormals give a signed zero, as the conversion does);
// results below the FP32 normal range, infinities and NaNs take the conversion instruction.
__device__ __forceinline__ float narrow(double x) {
  const unsigned hw = (unsigned)__double2hiint(x), lw = (unsigned)__double2loint(x);
  const unsigned E = (hw >> 20) & 0x7ffu;
  if (E == 0u) return __uint_as_float(hw & 0x80000000u);
  if (E - 897u > 253u) return (float)x;  // the float is not normal: subnormal, zero, inf, NaN
  const unsigned m = ((hw & 0xfffffu) << 3) | (lw >> 29);  // the 23 kept mantissa bits
  const unsigned rest = lw & 0x1fffffffu;                   // the 29 dropped ones
  unsigned r = ((E - 896u) << 23) | m;
  // round half to even; a carry out of the mantissa raises the exponent, which is the rounded
  // value (and infinity above the largest float)
  r += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
  return __uint_as_float((hw & 0x80000000u) | r);
}

// pair -> double: one FP64 addition.
__device__ __forceinline__ double to_double(f32x2 x) { return widen(x.hi) + widen(x.lo); }

// ---- arithmetic
__device__ __forceinline__ f32x2 operator-(f32x2 x) { return f32x2(-x.hi, -x.lo); }

__device__ __forceinline__ f32x2 operator+(f32x2 x, f32x2 y) {
  float sh, sl, zh, zl;
  two_sum(x.hi, y.hi, sh, sl);
  const float v = __fadd_rn(x.lo, y.lo);
  const float w = __fadd_rn(sl, v);
  fast_two_sum(sh, w, zh, zl);
  return f32x2(zh, zl);
}

__device__ __forceinline__ f32x2 operator-(f32x2 x, f32x2 y) { return x + (-y); }

__device__ __forceinline__ f32x2 operator*(f32x2 x, f32x2 y) {
  float ch, cl1, zh, zl;
  two_prod(x.hi, y.hi, ch, cl1);
  const float tl = __fmul_rn(x.hi, y.lo);
  const float cl2 = __fmaf_rn(x.lo, y.hi, tl);
  const float cl3 = __fadd_rn(cl1, cl2);
  fast_two_sum(ch, cl3, zh, zl);
  return f32x2(zh, zl);
}

// x / y: q0 = x.hi / y.hi in FP32, residual r = x - q0 y formed with TwoProd (x.hi - p is exact:
// p is within a few ulps of x.hi), q = q0 + r / y.hi.
__device__ __forceinline__ f32x2 operator/(f32x2 x, f32x2 y) {
  const float iy = __frcp_rn(y.hi);
  const float q0 = __fmul_rn(x.hi, iy);
  float p, pe;
  two_prod(q0, y.hi, p, pe);
  float r = __fsub_rn(__fsub_rn(x.hi, p), pe);
  r = __fadd_rn(r, __fmaf_rn(-q0, y.lo, x.lo));
  const float q1 = __fmul_rn(r, iy);
  float zh, zl;
  fast_two_sum(q0, q1, zh, zl);
  return f32x2(zh, zl);
}

__device__ __forceinline__ f32x2& operator+=(f32x2& x, f32x2 y) { return x = x + y; }
__device__ __forceinline__ f32x2& operator-=(f32x2& x, f32x2 y) { return x = x - y; }
__device__ __forceinline__ f32x2& operator*=(f32x2& x, f32x2 y) { return x = x * y; }

// ---- comparisons (normalised pairs: hi decides unless equal)
__device__ __forceinline__ bool operator<(f32x2 x, f32x2 y) { return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo); }
__device__ __forceinline__ bool operator>(f32x2 x, f32x2 y) { return y < x; }
__device__ __forceinline__ bool operator<=(f32x2 x, f32x2 y) { return !(y < x); }
__device__ __forceinline__ bool operator>=(f32x2 x, f32x2 y) { return !(x < y); }
__device__ __forceinline__ bool operator==(f32x2 x, f32x2 y) { return x.hi == y.hi && x.lo == y.lo; }
__device__ __forceinline__ bool operator!=(f32x2 x, f32x2 y) { return !(x == y); }

__device__ __forceinline__ f32x2 fabs(f32x2 x) { return x.hi < 0.0f ? -x : x; }
__device__ __forceinline__ f32x2 fmin(f32x2 x, f32x2 y) { return y < x ? y : x; }
__device__ __forceinline__ f32x2 fmax(f32x2 x, f32x2 y) { return x < y ? y : x; }

// sqrt(x) for x >= 0: s0 = sqrt(x.hi) in FP32, then s = s0 + (x - s0^2) / (2 s0) with the
// residual formed exactly.  sqrt(0) = 0.
__device__ __forceinline__ f32x2 sqrt(f32x2 x) {
  if (!(x.hi > 0.0f)) return f32x2(0.0f, 0.0f);
  const float rs = rsqrtf(x.hi);
  const float s0 = __fmul_rn(x.hi, rs);
  float p, pe;
  two_prod(s0, s0, p, pe);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p), pe), x.lo);
  const float c = __fmul_rn(__fmul_rn(r, rs), 0.5f);
  float zh, zl;
  fast_two_sum(s0, c, zh, zl);
  return f32x2(zh, zl);
}

// 1 / sqrt(x) for x > 0: y0 = rsqrt(x.hi) in FP32, then y = y0 + y0 (1 - x y0^2) / 2 with
// 1 - x y0^2 formed in double-word arithmetic.
__device__ __forceinline__ f32x2 rsqrt(f32x2 x) {
  const float y0 = rsqrtf(x.hi);
  float p, pe;
  two_prod(y0, y0, p, pe);
  const f32x2 e = f32x2(1.0f, 0.0f) - x * f32x2(p, pe);
  const float c = __fmul_rn(__fmul_rn(y0, e.hi), 0.5f);
  float zh, zl;
  fast_two_sum(y0, c, zh, zl);
  return f32x2(zh, zl);
}

}  // namespace dw
using dw::f32x2;

// Run-time conversions into the arithmetic type R of a kernel (plain casts for double and
// float; integer-based split for pairs) and back to double.
template <typename R>
struct Conv {
  template <typename S>
  static __device__ __forceinline__ R from(S x) { return (R)x; }
};
template <>
struct Conv<f32x2> {
  static __device__ __forceinline__ f32x2 from(double x) { return dw::split(x); }
};
template <typename R, typename S>
__device__ __forceinline__ R cvt(S x) { return Conv<R>::from(x); }
template <typename R, typename S>
__device__ __forceinline__ R ldc(const S* p) { return Conv<R>::from(__ldg(p)); }

__device__ __forceinline__ double to_dbl(double x) { return x; }
__device__ __forceinline__ double to_dbl(float x) { return dw::widen_exact(x); }
__device__ __forceinline__ double to_dbl(f32x2 x) { return dw::to_double(x); }

// A double stored in the element type T of an FP32 or FP64 result (integer rounding for FP32).
template <typename T>
__device__ __forceinline__ T store_as(double x) {
  if constexpr (sizeof(T) == sizeof(float)) return dw::narrow(x);
  else return x;
}

}  // namespace hzn
