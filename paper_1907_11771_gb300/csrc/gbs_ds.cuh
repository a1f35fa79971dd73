// FP32-pair ("double-single") arithmetic for the GBS_F32X2 precision.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2, about 48
// significant bits, computed with FP32 instructions only (GB300 runs FP64 at a small fraction
// of its FP32 rate).  Sums use Knuth's error-free TwoSum of the high parts plus the low parts,
// renormalised by Dekker's Fast2Sum; products use the FMA form of Dekker's TwoProd.  Relative
// error per operation is a small multiple of 2^-48 (about 4e-15), except that a sum of two
// nearly opposite values keeps an absolute error of that size relative to the operands.  The
// products go through __fmul_rn / fmaf so that the compiler cannot contract the rounded product
// into a later addition, which would break the error-free transformation.
#pragma once

#include <cuda_runtime.h>

namespace gbs {

struct __align__(8) dsf {
  float hi, lo;
  dsf() = default;
  __host__ __device__ constexpr dsf(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr dsf(int v) : hi(float(v)), lo(0.f) {}
  // nearest pair to a double: hi = fl(d), lo = fl(d - hi) (d - hi is exact in FP64)
  __host__ __device__ constexpr dsf(double d) : hi(float(d)), lo(float(d - double(float(d)))) {}
  __host__ __device__ explicit constexpr operator double() const { return double(hi) + double(lo); }
};

__device__ __forceinline__ dsf ds_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return dsf(s, (a - (s - bb)) + (b - bb));
}

__device__ __forceinline__ dsf ds_fast_two_sum(float a, float b) {   // needs |a| >= |b| or a == 0
  const float s = a + b;
  return dsf(s, b - (s - a));
}

__device__ __forceinline__ dsf operator+(dsf a, dsf b) {
  const dsf s = ds_two_sum(a.hi, b.hi);
  return ds_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ dsf operator-(dsf a) { return dsf(-a.hi, -a.lo); }
__device__ __forceinline__ dsf operator-(dsf a, dsf b) { return a + (-b); }
__device__ __forceinline__ dsf operator*(dsf a, dsf b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);   // exact rounding error of hi * hi
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return ds_fast_two_sum(p, e);
}
__device__ __forceinline__ dsf& operator+=(dsf& a, dsf b) { return a = a + b; }
__device__ __forceinline__ dsf& operator-=(dsf& a, dsf b) { return a = a - b; }
__device__ __forceinline__ dsf& operator*=(dsf& a, dsf b) { return a = a * b; }

// scaling by a power of two is exact
__device__ __forceinline__ dsf ds_scale2(dsf a, float pow2) { return dsf(a.hi * pow2, a.lo * pow2); }

__device__ __forceinline__ dsf ldg(const dsf* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return dsf(v.x, v.y);
}

// Gragg's average (y_(N-1) + 2 y_N + y_(N+1)) / 4 in pair arithmetic (the scalings are exact)
__device__ __forceinline__ dsf gragg_avg(dsf ym, dsf y0, dsf yp) {
  return ds_scale2((ym + yp) + ds_scale2(y0, 2.f), 0.25f);
}

}  // namespace gbs
