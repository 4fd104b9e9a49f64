// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// floats, about 48 significand bits. Error-free transformations after Knuth
// (TwoSum), Dekker (Fast2Sum) and the fused multiply-add product error
// (TwoProd); addition is the "sloppy" double-float sum without renormalisation
// (error about 2^-46 of |a| + |b|), multiplication keeps the cross terms hi*lo
// and renormalises (relative error about 2^-46).
//
// Used for the refinement residual of the mixed solve (FDE_MIXED_DF): GB300
// runs float arithmetic 58 times faster than double, and a double-float
// transform needs roughly ten float operations per double operation.
#pragma once
#include <cuda_runtime.h>

namespace fde {

struct __align__(8) dd {
  float hi, lo;
  __host__ __device__ constexpr dd() : hi(0.f), lo(0.f) {}
  __host__ __device__ constexpr dd(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
};

__device__ __forceinline__ dd dd_fast2sum(float a, float b) {
  const float s = a + b;
  return dd(s, b - (s - a));
}

// Sum without the final renormalisation: hi is the float sum of the high parts,
// lo collects its exact rounding error (TwoSum) and the low parts. The pair is
// an unevaluated sum whose lo may exceed half an ulp of hi; products renormalise
// (operator*), and in the transforms every product has one normalised factor (a
// twiddle or a symbol value), so the norm-wise error stays near 2^-46.
__device__ __forceinline__ dd operator+(dd a, dd b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb);
  return dd(s, e + (a.lo + b.lo));
}

__host__ __device__ constexpr dd operator-(dd a) { return dd(-a.hi, -a.lo); }
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }

__device__ __forceinline__ dd operator*(dd a, dd b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return dd_fast2sum(p, e);
}

__device__ __forceinline__ dd& operator+=(dd& a, dd b) { return a = a + b; }
__device__ __forceinline__ dd& operator*=(dd& a, dd b) { return a = a * b; }

struct __align__(16) dd2 {
  dd x, y;
};

// conversions between the storage type (double) and the compute type
__device__ __forceinline__ dd to_dd(double v) {
  const float h = __double2float_rn(v);
  return dd(h, __double2float_rn(v - (double)h));
}
__device__ __forceinline__ double to_double(dd v) { return (double)v.hi + (double)v.lo; }

}  // namespace fde
