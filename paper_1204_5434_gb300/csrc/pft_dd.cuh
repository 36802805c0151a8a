// pft_dd.cuh -- double-float arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2: about 48
// significant bits, against 53 for an IEEE double, with the float exponent range.  GB300
// runs FP64 at 1/64 of its FP32 rate, so an FFT in double-float arithmetic (a dozen FP32
// operations per FP64 operation) can outrun the same FFT in FP64.
//
// Building blocks (all error-free transformations in round-to-nearest):
//   TwoSum(a, b)     = (s, e) with s = fl(a + b), s + e = a + b exactly (Knuth; 6 flops)
//   Fast2Sum(a, b)   = the same for |a| >= |b| (Dekker; 3 flops)
//   TwoProd(a, b)    = (p, e) with p = fl(a b), p + e = a b exactly: e = fma(a, b, -p)
// Double-word sum: TwoSum of the high parts, the low parts added to the error, one
// Fast2Sum to renormalise (the "sloppy" double-word sum; its error is below about
// 2u^2 (|x| + |y|) with u = 2^-24, a bound relative to the operands rather than to the
// sum, which is the normwise bound the error analysis of an FFT uses).  Double-word
// product: TwoProd of the high parts, the cross products added by FMA, one Fast2Sum
// (relative error below 5u^2).  Both are analysed in Joldes, Muller and Popescu, "Tight
// and rigorous error bounds for basic building blocks of double-word arithmetic", ACM
// TOMS 44 (2017).
// The high product uses __fmul_rn so that the compiler never contracts it into a later
// addition: the error-free transformations need every operation rounded on its own.
#pragma once
#include <cuda_runtime.h>

#include "pft_fft.cuh"

namespace pft {

struct __align__(8) dd {
  float hi, lo;
  __host__ __device__ constexpr dd() : hi(0.f), lo(0.f) {}
  __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
  // From a double (constants of the transforms, folded at compile time; tables on the host).
  __host__ __device__ constexpr dd(double c) : hi((float)c), lo((float)(c - (double)(float)c)) {}
  __host__ __device__ constexpr dd(int c) : hi((float)c), lo(0.f) {}
};

__device__ __forceinline__ dd dd_fast2sum(float a, float b) {
  const float s = a + b;
  return dd(s, b - (s - a));
}

__device__ __forceinline__ dd operator+(dd a, dd b) {
  const float s = a.hi + b.hi;
  const float bp = s - a.hi;
  float e = (a.hi - (s - bp)) + (b.hi - bp);
  e += a.lo + b.lo;
  return dd_fast2sum(s, e);
}
__device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }
__device__ __forceinline__ dd operator*(dd a, dd b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return dd_fast2sum(p, e);
}
__device__ __forceinline__ dd& operator+=(dd& a, dd b) { return a = a + b; }
__device__ __forceinline__ dd& operator-=(dd& a, dd b) { return a = a - b; }
__device__ __forceinline__ dd& operator*=(dd& a, dd b) { return a = a * b; }

struct __align__(16) dd2 {
  dd x, y;
};
template <> struct cpx_t<dd> { using type = dd2; };

// Complex double-word product with one renormalisation per component: the two exact high
// products and their errors, TwoSum of the high products, every lower-order term added to
// the error, Fast2Sum.  (Re = a.x b.x - a.y b.y, Im = a.x b.y + a.y b.x.)
__device__ __forceinline__ dd dd_dot2(dd a, dd b, dd c, dd d) {  // a b + c d
  const float p = __fmul_rn(a.hi, b.hi);
  const float q = __fmul_rn(c.hi, d.hi);
  float ep = fmaf(a.hi, b.hi, -p);
  float eq = fmaf(c.hi, d.hi, -q);
  const float s = p + q;
  const float bp = s - p;
  float e = (p - (s - bp)) + (q - bp);
  ep = fmaf(a.hi, b.lo, ep);
  ep = fmaf(a.lo, b.hi, ep);
  eq = fmaf(c.hi, d.lo, eq);
  eq = fmaf(c.lo, d.hi, eq);
  e += ep + eq;
  return dd_fast2sum(s, e);
}
template <> __device__ __forceinline__ dd2 cmul<dd2>(dd2 a, dd2 b) {
  dd2 r;
  r.x = dd_dot2(a.x, b.x, -a.y, b.y);
  r.y = dd_dot2(a.x, b.y, a.y, b.x);
  return r;
}
template <> __device__ __forceinline__ dd2 cmulc<dd2>(dd2 a, dd2 b) {
  dd2 r;
  r.x = dd_dot2(a.x, b.x, a.y, b.y);
  r.y = dd_dot2(a.y, b.x, -a.x, b.y);
  return r;
}

// double <-> double-float.  The split rounds hi to the nearest float and keeps the
// remainder rounded to a float (the FP64 pipe does the subtraction: used once per march
// for q_0 and on the host for the tables).  The sum back to double widens both parts on
// the integer pipe and adds them in one FP64 addition.
__device__ __forceinline__ dd dd_from_double(double x) {
  const float h = __double2float_rn(x);
  return dd(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ double dd_to_double(dd a) { return widen(a.hi) + widen(a.lo); }
inline dd dd_split_host(double x) {
  const float h = (float)x;
  return dd(h, (float)(x - (double)h));
}

}  // namespace pft
