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

namespace gbs {

// Two independent pair values processed together with packed FP32-pair instructions
// (f32x2): lane x is one value, lane y the other.  Same algorithms as dsf, lane by lane.
struct ds2 {
  float2 hi, lo;
};

__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) { return __fadd2_rn(a, b); }

// TwoSum lane by lane, then the low parts, then Fast2Sum
__device__ __forceinline__ ds2 operator+(const ds2& a, const ds2& b) {
  const float2 s = f2_add(a.hi, b.hi);
  const float2 bb = f2_sub(s, a.hi);
  const float2 e = f2_add(f2_sub(a.hi, f2_sub(s, bb)), f2_sub(b.hi, bb));
  const float2 t = f2_add(e, f2_add(a.lo, b.lo));
  const float2 h = f2_add(s, t);
  return ds2{h, f2_sub(t, f2_sub(h, s))};
}
__device__ __forceinline__ ds2 operator-(const ds2& a, const ds2& b) {
  const float2 s = f2_sub(a.hi, b.hi);
  const float2 bb = f2_sub(s, a.hi);                 // the rounded -b.hi
  const float2 e = f2_sub(f2_sub(a.hi, f2_sub(s, bb)), f2_add(b.hi, bb));
  const float2 t = f2_add(e, f2_sub(a.lo, b.lo));
  const float2 h = f2_add(s, t);
  return ds2{h, f2_sub(t, f2_sub(h, s))};
}

// (value pair) times one pair constant c = chi + clo on both lanes (FMA TwoProd)
__device__ __forceinline__ ds2 ds2_mul(const ds2& a, float chi, float clo) {
  const float2 ch = make_float2(chi, chi), nch = make_float2(-chi, -chi);
  const float2 q = __fmul2_rn(nch, a.hi);             // -(chi * a.hi) rounded
  float2 e = __ffma2_rn(ch, a.hi, q);                 // its exact error
  e = __ffma2_rn(ch, a.lo, e);
  if (clo != 0.f) e = __ffma2_rn(make_float2(clo, clo), a.hi, e);
  const float2 h = f2_sub(e, q);                       // p + e with p = -q
  return ds2{h, f2_sub(e, f2_add(h, q))};
}

// lane-wise product with a per-lane pair multiplier (m.hi, m.lo lanes)
__device__ __forceinline__ ds2 ds2_mul(const ds2& a, const ds2& m) {
  const float2 nmh = make_float2(-m.hi.x, -m.hi.y);
  const float2 q = __fmul2_rn(nmh, a.hi);
  float2 e = __ffma2_rn(m.hi, a.hi, q);
  e = __ffma2_rn(m.hi, a.lo, e);
  e = __ffma2_rn(m.lo, a.hi, e);
  const float2 h = f2_sub(e, q);
  return ds2{h, f2_sub(e, f2_add(h, q))};
}

__device__ __forceinline__ dsf lane_x(const ds2& a) { return dsf(a.hi.x, a.lo.x); }
__device__ __forceinline__ dsf lane_y(const ds2& a) { return dsf(a.hi.y, a.lo.y); }
__device__ __forceinline__ ds2 make_ds2(dsf x, dsf y) { return ds2{make_float2(x.hi, y.hi), make_float2(x.lo, y.lo)}; }

// Centred finite-difference sums of two pair lanes with the weights as integers over a common
// divisor: sum_j m_j (a[+j] - a[-j]) = div x the stencil sum (4th order: m = 8, -1, div 12; 6th
// order: 45, -9, 1, div 60); the caller folds 1/div into a scaling it applies anyway.  hi(j) and
// lo(j) give the two lanes' hi and lo parts at offset j.  The hi parts' differences are taken
// exactly (TwoDiff), the integer products exactly (FMA error term; 8 and 1 need none), the main
// terms are summed exactly (TwoSum), and every small term -- the differences' errors, the lo
// parts' differences, the products' errors, the sums' errors -- goes into one FP32 accumulator,
// whose own rounding is 2^-24 of terms already 2^-24 below the result: the pair carries about 48
// bits as the general pair operations do, for about two thirds of their instructions.
template <int R>
__host__ __device__ constexpr float fd_int(int j) {
  return R == 2 ? (j == 1 ? 8.f : -1.f) : (j == 1 ? 45.f : j == 2 ? -9.f : 1.f);
}
template <int R>
__host__ __device__ constexpr double fd_div() { return R == 2 ? 12.0 : 60.0; }

template <int R, class Hi, class Lo>
__device__ __forceinline__ ds2 isum_x2(Hi hi, Lo lo) {
  float2 S = make_float2(0.f, 0.f), small = make_float2(0.f, 0.f);
#pragma unroll
  for (int j = 1; j <= R; ++j) {
    const float2 a = hi(j), b = hi(-j);
    const float2 d = f2_sub(a, b);                                   // TwoDiff: d + e = a - b
    const float2 bb = f2_sub(d, a);
    const float2 e = f2_sub(f2_sub(a, f2_sub(d, bb)), f2_add(b, bb));
    const float2 l = f2_sub(lo(j), lo(-j));
    const float m = fd_int<R>(j);   // folds: the loop is unrolled
    const float2 mm = make_float2(m, m);
    float2 pm;
    if (m == 1.f || m == -1.f || m == 8.f) {                         // exact products
      pm = m == 1.f ? d : __fmul2_rn(mm, d);
    } else {
      pm = __fmul2_rn(mm, d);
      small = f2_add(small, __ffma2_rn(mm, d, make_float2(-pm.x, -pm.y)));   // product error
    }
    small = __ffma2_rn(mm, f2_add(e, l), small);
    if (j == 1) {
      S = pm;
    } else {                                                          // TwoSum S + pm
      const float2 t = f2_add(S, pm);
      const float2 tb = f2_sub(t, S);
      small = f2_add(small, f2_add(f2_sub(S, f2_sub(t, tb)), f2_sub(pm, tb)));
      S = t;
    }
  }
  const float2 h = f2_add(S, small);                                 // Fast2Sum
  return ds2{h, f2_sub(small, f2_sub(h, S))};
}

}  // namespace gbs
