// Periodic centred finite-difference stencils and the wave right-hand sides,
// as device functions over global memory (point-parallel kernels).
//
// First derivative, radius R (order 2R), antisymmetric weights a_j:
//   (D f)_i = (1/dx) sum_{j=1..R} a_j (f_{i+j} - f_{i-j})
//   R = 2 (order 4): a = (2/3, -1/12)
//   R = 3 (order 6): a = (3/4, -3/20, 1/60)
// Systems (f(y) = A y):
//   1D wave:   f_u = D v, f_v = D u
//   acoustics: f_p = -kappa sum_d D_d u_d,  f_{u_d} = -b D_d p   (b = 1/rho)
// Transposed operator (D_d^T = -D_d on a periodic grid):
//   (A^T l)_p = sum_d D_d (b l_{u_d}),  (A^T l)_{u_d} = D_d (kappa l_p)
#pragma once

#include <cstdint>

namespace gbs {

enum { SYS_WAVE1D = 1, SYS_ACOUSTIC = 2 };

template <int R>
__host__ __device__ constexpr double fd_coef(int j) {
  return R == 2 ? (j == 1 ? 2.0 / 3.0 : -1.0 / 12.0)
                : (j == 1 ? 0.75 : (j == 2 ? -0.15 : 1.0 / 60.0));
}

template <int SYS, int DIM>
__host__ __device__ constexpr int n_fields() {
  return SYS == SYS_WAVE1D ? 2 : 1 + DIM;
}

template <typename T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

// Gragg's average (y_(N-1) + 2 y_N + y_(N+1)) / 4 rounded once.  In FP32 the two additions
// are carried as exact sum/error pairs (Knuth's TwoSum), so the result is the FP32 rounding of
// the exact average without touching the (slow) FP64 pipe.
__device__ __forceinline__ float gragg_avg(float ym, float y0, float yp) {
  const float s = ym + yp;
  const float bs = s - ym;
  const float es = (ym - (s - bs)) + (yp - bs);
  const float y2 = 2.f * y0;
  const float t = s + y2;
  const float bt = t - s;
  const float et = (s - (t - bt)) + (y2 - bt);
  return (t + (es + et)) * 0.25f;
}
__device__ __forceinline__ double gragg_avg(double ym, double y0, double yp) {
  return (ym + 2.0 * y0 + yp) * 0.25;
}

// (sh, sl) += (c_hi + c_lo) * y in FP32 pairs: TwoProd of c_hi * y by one FMA, c_lo * y added to
// its error, TwoSum into the running pair.  Error about 2^-48 of the sum of |c y| terms, using
// FP32 units only (the _rn intrinsics keep the compiler from contracting the error terms).
__device__ __forceinline__ void pair_combine_add(float c_hi, float c_lo, float y, float& sh, float& sl) {
  const float p = __fmul_rn(c_hi, y);
  const float pe = fmaf(c_lo, y, fmaf(c_hi, y, -p));
  const float t = __fadd_rn(sh, p);
  const float bv = __fsub_rn(t, sh);
  const float te = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bv)), __fsub_rn(p, bv));
  sl = __fadd_rn(sl, __fadd_rn(te, pe));
  sh = __fadd_rn(t, sl);
  sl = __fsub_rn(sl, __fsub_rn(sh, t));
}

// FP32 states are advanced in increment form: every sequence carries d_n = y_n - y_0 instead of
// y_n, with f(y_n) = f0 + A d_n (f is linear), so
//   d_0 = 0,  d_1 = h f0,  d_(n+1) = d_(n-1) + 2h f0 + 2h A d_n,  d* = (d_(N-1) + 2 d_N + d_(N+1)) / 4
// and y(t + H) = y_0 + sum_k c_k d*_k (sum_k c_k = 1).  This is the same linear map as Sec. 2.1
// eq. "GBS"; in FP32 each rounding is then relative to |d| rather than |y|, and the combine's
// large alternating weights amplify those roundings, so the increment form lowers the FP32
// error several-fold (a textbook device for extrapolation methods).  The FP64 and FP32-pair
// paths keep the plain form.
//
// h = hi + lo: a double split into two floats (the FP32 kernels' step sizes).
__host__ __device__ __forceinline__ void split_h(double h, float& hi, float& lo) {
  hi = (float)h;
  lo = (float)(h - (double)hi);
}
// fl(h f) for h = hi + lo: TwoProd of hi f by one FMA plus lo f, so the result is within about
// one ulp of the exact product; a step size rounded to FP32 would instead scale every point of
// a sequence by the same wrong factor, an error that adds up coherently over macro-steps.
__device__ __forceinline__ float mul_split(float hi, float lo, float f) {
  const float p = __fmul_rn(hi, f);
  const float e = fmaf(hi, f, -p);
  return __fadd_rn(p, fmaf(lo, f, e));
}

// mul_split on a packed pair of lanes (Blackwell f32x2 instructions): each lane as mul_split
__device__ __forceinline__ float2 mul_split2(float2 hi, float2 lo, float2 f) {
  const float2 p = __fmul2_rn(hi, f);
  const float2 e = __ffma2_rn(hi, f, make_float2(-p.x, -p.y));
  return __fadd2_rn(p, __ffma2_rn(lo, f, e));
}

// Exact FP32 -> FP64 promotion on the integer pipe, bit for bit the hardware conversion for every
// float but the signalling NaNs (all 2^32 inputs compared with it on the device by
// gbs_selftest_f32_to_f64): a normal float's sign, exponent (re-biased by 1023 - 127 = 896) and
// 23 mantissa bits placed into the double's fields; infinities and NaNs keep exponent 2047 and
// their payload (the conversion also sets a signalling NaN's quiet bit; an FMA on either gives a
// NaN); a subnormal m 2^-149 is normalised (its leading bit found by clz); zero keeps its sign.
// GB300's conversion instruction shares the slow FP64 pipe with the combine's FMAs, so a
// converted operand per FMA would double that pipe's work.
__device__ __forceinline__ double promote(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned sign = b & 0x80000000u, mag = b & 0x7fffffffu, ex = mag >> 23;
  unsigned hi = sign | ((mag >> 3) + (ex == 0xffu ? (1792u << 20) : (896u << 20)));
  unsigned lo = b << 29;
  if (ex == 0u) {
    const int sh = __clz(mag) - 8;                     // mag << sh has bit 23 set (mag != 0)
    const unsigned fr = (mag << sh) & 0x7fffffu;
    hi = mag ? (sign | ((897u - (unsigned)sh) << 20) | (fr >> 3)) : sign;
    lo = mag ? (fr << 29) : 0u;
  }
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ double to_f64(float f) { return promote(f); }
template <typename T>
__device__ __forceinline__ double to_f64(T v) { return (double)v; }

// The combine of the plain path's last leap-frog step of sequence k: y_out (+)= c_k y*_k in FP64.
// FP32 states are in increment form (y*_k = y_0 + d*_k): the first sequence starts the
// accumulator at y_0, each adds c_k d*_k (d*_k promoted exactly), the last rounds once to FP32.
// kIntPromote: FP32 inputs promoted on the integer pipe (promote) instead of by the conversion
// instruction on the FP64 pipe; measured faster in the 3D kernels (1.4% per 3D macro-step) and
// slower in the 2D ones (0.6%), whose issue slots are the scarcer resource.
template <typename T, typename O, bool kIntPromote = false>
__device__ __forceinline__ void combine_last(double* acc, int64_t e, bool first, bool last, double c, T ystar,
                                             O* yo, T y0 = T(0)) {
  auto f64 = [](T v) -> double {
    if constexpr (kIntPromote) return to_f64(v);
    else return (double)v;
  };
  const double ys = f64(ystar);
  double a2;
  if constexpr (sizeof(T) == 4 && sizeof(O) == 4) a2 = fma(c, ys, first ? f64(y0) : acc[e]);
  else a2 = first ? c * ys : fma(c, ys, acc[e]);
  if (last) yo[e] = static_cast<O>(a2);
  else acc[e] = a2;
}

// Geometry of one point inside one problem.
struct PointGeo {
  int64_t i;        // flat point index inside the problem
  int c[3];         // coordinates (x, y, z)
  int n[3];         // sizes
  int64_t st[3];    // strides (1, nx, nx*ny)
};

__device__ __forceinline__ int64_t nb_off(int c, int j, int n, int64_t st) {
  int cj = c + j;
  if (cj >= n) cj -= n;
  else if (cj < 0) cj += n;
  return (int64_t)(cj - c) * st;
}

// D_d f at the point (read-only input f).  Interior points use fixed offsets; only points
// within R of the periodic boundary wrap.
template <typename T, int R>
__device__ __forceinline__ T dstencil(const T* __restrict__ f, const PointGeo& g, int d, T inv_dx) {
  const T* p = f + g.i;
  const int c = g.c[d], n = g.n[d];
  const int64_t st = g.st[d];
  T s = T(0);
  if (c >= R && c < n - R) {
#pragma unroll
    for (int j = 1; j <= R; ++j) s += T(fd_coef<R>(j)) * (ldg(p + j * st) - ldg(p - j * st));
  } else {
#pragma unroll
    for (int j = 1; j <= R; ++j)
      s += T(fd_coef<R>(j)) * (ldg(p + nb_off(c, j, n, st)) - ldg(p + nb_off(c, -j, n, st)));
  }
  return s * inv_dx;
}

// D_d (w * f) at the point, w a media array (for the transposed operator).
template <typename T, int R>
__device__ __forceinline__ T dstencil_w(const T* __restrict__ f, const T* __restrict__ w,
                                        const PointGeo& g, int d, T inv_dx) {
  T s = T(0);
#pragma unroll
  for (int j = 1; j <= R; ++j) {
    const int64_t op = nb_off(g.c[d], j, g.n[d], g.st[d]);
    const int64_t om = nb_off(g.c[d], -j, g.n[d], g.st[d]);
    s += T(fd_coef<R>(j)) * (ldg(w + g.i + op) * ldg(f + g.i + op) - ldg(w + g.i + om) * ldg(f + g.i + om));
  }
  return s * inv_dx;
}

// f(y) at the point; y points to the problem's state block, fields P apart.
template <typename T, int SYS, int DIM, int R>
__device__ __forceinline__ void rhs_point(const T* __restrict__ y, int64_t P, const PointGeo& g,
                                          const T* inv_dx, T kap, T bb, T* f) {
  if (SYS == SYS_WAVE1D) {
    f[0] = dstencil<T, R>(y + P, g, 0, inv_dx[0]);
    f[1] = dstencil<T, R>(y, g, 0, inv_dx[0]);
  } else {
    T div = T(0);
#pragma unroll
    for (int d = 0; d < DIM; ++d) div += dstencil<T, R>(y + (1 + d) * P, g, d, inv_dx[d]);
    f[0] = -kap * div;
#pragma unroll
    for (int d = 0; d < DIM; ++d) f[1 + d] = -bb * dstencil<T, R>(y, g, d, inv_dx[d]);
  }
}

// div u of the acoustic state at the point.
template <typename T, int DIM, int R>
__device__ __forceinline__ T div_point(const T* __restrict__ y, int64_t P, const PointGeo& g,
                                       const T* inv_dx) {
  T div = T(0);
#pragma unroll
  for (int d = 0; d < DIM; ++d) div += dstencil<T, R>(y + (1 + d) * P, g, d, inv_dx[d]);
  return div;
}

// A^T l at the point for acoustics.
template <typename T, int DIM, int R>
__device__ __forceinline__ void rhs_T_point(const T* __restrict__ l, int64_t P, const PointGeo& g,
                                            const T* inv_dx, const T* __restrict__ kappa,
                                            const T* __restrict__ b, T* f) {
  T s = T(0);
#pragma unroll
  for (int d = 0; d < DIM; ++d) s += dstencil_w<T, R>(l + (1 + d) * P, b, g, d, inv_dx[d]);
  f[0] = s;
#pragma unroll
  for (int d = 0; d < DIM; ++d) f[1 + d] = dstencil_w<T, R>(l, kappa, g, d, inv_dx[d]);
}

}  // namespace gbs
