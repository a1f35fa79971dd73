// Point-parallel ("plain") GBS kernels: one kernel per Forward-Euler or
// leap-frog step, one thread per grid point, neighbours read through the
// read-only cache.  This is the unfused path, used for FP64 and as the
// baseline the time-blocked FP32 kernels are measured against.
//
// One macro-step (Sec. 2.1 eq. "GBS", Sec. 3.6, Sec. 3.2):
//   k_f0             f0 = f(y_in)                       shared first evaluation
//   for each sequence index k:
//     k_fe(k)        L1 = y_in + h_k f0                 Forward Euler
//     k_lf(k, n)     n = 1..N_k-1: y_(n+1) = y_(n-1) + 2 h_k f(y_n)   (in place over y_(n-1))
//                    n = N_k: y_(N+1), averaging and the FP64 combine
//                    acc (+)= c_k y*_k, the last sequence writing y_out
// With a batch, every launch covers all problems; a problem whose scheme has
// no step (k, n) leaves the launch at once.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <type_traits>

#include "gbs_ds.cuh"
#include "gbs_internal.h"
#include "gbs_seqfuse.h"
#include "gbs_stencil.cuh"

namespace gbs {

// Element type of the caller's output state for a level type: FP32 pairs hand back FP64.
template <typename T>
struct out_of {
  using type = T;
};
template <>
struct out_of<dsf> {
  using type = double;
};

namespace {

struct Loc {
  int prob;
  int64_t i;
};

// Map this thread to (problem, point); prob = -1 when past the problem's end.
__device__ __forceinline__ Loc locate(const StepPlan& p) {
  int lo = 0, hi = p.batch - 1;
  const int64_t blk = blockIdx.x;
  while (lo < hi) {  // last problem with blk_begin <= blk
    const int mid = (lo + hi + 1) >> 1;
    if (p.probs[mid].blk_begin <= blk) lo = mid;
    else hi = mid - 1;
  }
  Loc L;
  L.prob = lo;
  L.i = (blk - p.probs[lo].blk_begin) * kPlainBlock + threadIdx.x;
  if (L.i >= p.probs[lo].pts) L.prob = -1;
  return L;
}

// Coordinates of flat point i (problems hold fewer than 2^31 points, so 32-bit
// unsigned division suffices).
__device__ __forceinline__ PointGeo geo_of(const ProbDev& q, int64_t i) {
  PointGeo g;
  g.i = i;
  g.n[0] = q.n[0];
  g.n[1] = q.n[1];
  g.n[2] = q.n[2];
  g.st[0] = 1;
  g.st[1] = q.n[0];
  g.st[2] = (int64_t)q.n[0] * q.n[1];
  const unsigned ui = (unsigned)i, nx = (unsigned)q.n[0], ny = (unsigned)q.n[1];
  const unsigned r = ui / nx;
  g.c[0] = (int)(ui - r * nx);
  const unsigned z = r / ny;
  g.c[1] = (int)(r - z * ny);
  g.c[2] = (int)z;
  return g;
}

// (h_k, 2 h_k) in the state type, without FP64 arithmetic on the FP32 path.
template <typename T>
__device__ __forceinline__ void step_sizes(const StepPlan& p, int prob, int k, T& h, T& h2) {
  const int i = prob * GBS_MAX_SEQ + k;
  if (sizeof(T) == 4) {
    const float2 v = p.hkf[i];
    h = T(v.x);
    h2 = T(v.y);
  } else {
    const double d = p.hk[i];
    h = T(d);
    h2 = T(2.0 * d);
  }
}

template <typename T>
__device__ __forceinline__ void load_inv_dx(const ProbDev& q, T* inv_dx) {
  inv_dx[0] = T(q.inv_dx[0]);
  inv_dx[1] = T(q.inv_dx[1]);
  inv_dx[2] = T(q.inv_dx[2]);
}

// FP32 right-hand sides in integer-weight form: the stencil weights as integers over a common
// divisor (fd_int, fd_div), so t = div dx_0 f(y) carries no rounded coefficient; the caller
// applies 1 / (div dx_0), times 2h in a leap-frog update, as a constant split into two floats
// (mul_split, or two FMAs), so that no rounding is shared by every point of a sequence (such a
// rounding perturbs the operator coherently, and modes near the stability limit amplify it).
// rr[d] = dx_0 / dx_d (ProbDev::rr; 1 for equal spacings).
template <int R>
__device__ __forceinline__ float isum_point(const float* __restrict__ f, const PointGeo& g, int d) {
  float s = 0.f;
#pragma unroll
  for (int j = 1; j <= R; ++j)
    s = fmaf(fd_int<R>(j), ldg(f + g.i + nb_off(g.c[d], j, g.n[d], g.st[d])) - ldg(f + g.i + nb_off(g.c[d], -j, g.n[d], g.st[d])), s);
  return s;
}
template <int SYS, int DIM, int R>
__device__ __forceinline__ void rhs_point_int(const float* __restrict__ y, int64_t P, const PointGeo& g,
                                              const float* rr, float kap, float bb, float* t) {
  if (SYS == SYS_WAVE1D) {
    t[0] = isum_point<R>(y + P, g, 0);
    t[1] = isum_point<R>(y, g, 0);
  } else {
    float sdiv = 0.f;
#pragma unroll
    for (int d = 0; d < DIM; ++d) sdiv = fmaf(rr[d], isum_point<R>(y + (1 + d) * P, g, d), sdiv);
    t[0] = -kap * sdiv;
#pragma unroll
    for (int d = 0; d < DIM; ++d) t[1 + d] = -bb * (rr[d] * isum_point<R>(y, g, d));
  }
}

template <typename T, int SYS, int DIM, int R>
__global__ void __launch_bounds__(kPlainBlock) k_f0(const StepPlan p, const T* __restrict__ y_in) {
  const Loc L = locate(p);
  if (L.prob < 0) return;
  const ProbDev& q = p.probs[L.prob];
  const PointGeo g = geo_of(q, L.i);
  constexpr int F = n_fields<SYS, DIM>();
  T inv_dx[3];
  load_inv_dx(q, inv_dx);
  T kap = T(0), bb = T(0);
  if (SYS == SYS_ACOUSTIC) {
    kap = ldg(static_cast<const T*>(p.kappa) + q.media_off + L.i);
    bb = ldg(static_cast<const T*>(p.b) + q.media_off + L.i);
  }
  T f[kMaxFields];
  if constexpr (std::is_same<T, float>::value) {
    float t[kMaxFields];
    rhs_point_int<SYS, DIM, R>(y_in + q.state_off, q.pts, g, q.rr, kap, bb, t);
#pragma unroll
    for (int fl = 0; fl < F; ++fl) f[fl] = mul_split(q.f0s[0], q.f0s[1], t[fl]);
  } else {
    rhs_point<T, SYS, DIM, R>(y_in + q.state_off, q.pts, g, inv_dx, kap, bb, f);
  }
  T* f0 = static_cast<T*>(p.f0) + q.state_off;
  if constexpr (SYS == SYS_ACOUSTIC && DIM == 2 && std::is_same<T, float>::value) {
    if (p.f0_aux) {
      p.f0_aux[q.media_off + L.i] = make_float4(kap, bb, f[0], f[1]);
      f0[2 * q.pts + L.i] = f[2];
      return;
    }
  }
#pragma unroll
  for (int fl = 0; fl < F; ++fl) f0[fl * q.pts + L.i] = f[fl];
}

template <typename T, int SYS, int DIM>
__global__ void __launch_bounds__(kPlainBlock) k_fe(const StepPlan p, const T* __restrict__ y_in, int k) {
  const Loc L = locate(p);
  if (L.prob < 0) return;
  const ProbDev& q = p.probs[L.prob];
  const SlotDev& s = p.slots[q.slot];
  if (k >= s.m) return;
  constexpr int F = n_fields<SYS, DIM>();
  T h, h2;
  step_sizes(p, L.prob, k, h, h2);
  const T* f0 = static_cast<const T*>(p.f0) + q.state_off;
  T* L1 = static_cast<T*>(p.L1) + q.state_off;
  const T* y0 = y_in + q.state_off;
  if constexpr (std::is_same<T, float>::value) {
    // increment form: d_1 = h f0 = (2h f0) / 2 (y_0 is added back by the combine)
    const float4 hq = p.hkq[L.prob * GBS_MAX_SEQ + k];
#pragma unroll
    for (int fl = 0; fl < F; ++fl) {
      const int64_t e = fl * q.pts + L.i;
      L1[e] = 0.5f * mul_split(hq.x, hq.y, f0[e]);
    }
  } else {
#pragma unroll
    for (int fl = 0; fl < F; ++fl) {
      const int64_t e = fl * q.pts + L.i;
      L1[e] = y0[e] + h * f0[e];
    }
  }
}

template <typename T, int SYS, int DIM, int R>
__global__ void __launch_bounds__(kPlainBlock) k_lf(const StepPlan p, const T* y_in, typename out_of<T>::type* y_out,
                                                     int k, int n) {
  const Loc L = locate(p);
  if (L.prob < 0) return;
  const ProbDev& q = p.probs[L.prob];
  const SlotDev& s = p.slots[q.slot];
  if (k >= s.m) return;
  const int N = s.steps[k];
  if (n > N) return;
  constexpr int F = n_fields<SYS, DIM>();
  T h, h2;
  step_sizes(p, L.prob, k, h, h2);
  T* const L0 = static_cast<T*>(p.L0) + q.state_off;
  T* const L1 = static_cast<T*>(p.L1) + q.state_off;
  const T* cur = (n & 1) ? L1 : L0;
  T* dst = (n & 1) ? L0 : L1;                          // y_(n+1) overwrites y_(n-1)
  const T* prev = (n == 1) ? (y_in + q.state_off) : dst;
  const PointGeo g = geo_of(q, L.i);
  T inv_dx[3];
  load_inv_dx(q, inv_dx);
  T kap = T(0), bb = T(0);
  if (SYS == SYS_ACOUSTIC) {
    kap = ldg(static_cast<const T*>(p.kappa) + q.media_off + L.i);
    bb = ldg(static_cast<const T*>(p.b) + q.media_off + L.i);
  }
  // FP32: increment form, d_(n+1) = d_(n-1) + 2h f0 + 2h A d_n with d_0 = 0, the right-hand side
  // in integer-weight form scaled by 2h / (div dx_0) as a float pair
  constexpr bool kInc = std::is_same<T, float>::value;
  T f[kMaxFields];
  float gh = 0.f, gl = 0.f, sch = 0.f, scl = 0.f;
  if constexpr (kInc) {
    const float4 hq = p.hkq[L.prob * GBS_MAX_SEQ + k];
    gh = hq.x;
    gl = hq.y;
    sch = hq.z;
    scl = hq.w;
    rhs_point_int<SYS, DIM, R>(cur, q.pts, g, q.rr, kap, bb, f);
  } else {
    rhs_point<T, SYS, DIM, R>(cur, q.pts, g, inv_dx, kap, bb, f);
  }
  // the leap-frog update prev + 2h f (FP32: the pair scaling of the integer-weight form)
  auto lf_update = [&](T pv, T fv) -> T {
    if constexpr (kInc) return fmaf(sch, fv, fmaf(scl, fv, pv));
    else return pv + h2 * fv;
  };
  const T* f0 = static_cast<const T*>(p.f0) + q.state_off;
  T pv[kMaxFields];
#pragma unroll
  for (int fl = 0; fl < F; ++fl) {
    const int64_t e = fl * q.pts + L.i;
    if constexpr (kInc) pv[fl] = (n == 1 ? T(0) : prev[e]) + mul_split(gh, gl, f0[e]);
    else pv[fl] = prev[e];
  }
  if (n < N) {
#pragma unroll
    for (int fl = 0; fl < F; ++fl) {
      const int64_t e = fl * q.pts + L.i;
      dst[e] = lf_update(pv[fl], f[fl]);
    }
    return;
  }
  // n == N: y_(N+1), averaging y* = (y_(N-1) + 2 y_N + y_(N+1)) / 4 in the state type,
  // then the FP64 combine.
  const double c = s.c[k];
  bool first, last;
  seq_first_last(p, k, s.m, first, last);
  double* acc = p.acc + q.state_off;
  auto* yo = y_out + q.state_off;
#pragma unroll
  for (int fl = 0; fl < F; ++fl) {
    const int64_t e = fl * q.pts + L.i;
    const T ym = kInc && n == 1 ? T(0) : prev[e];
    const T y0 = cur[e];
    const T yp = lf_update(pv[fl], f[fl]);
    combine_last(acc, e, first, last, c, gragg_avg(ym, y0, yp), yo,
                 kInc && first && !p.partial ? y_in[q.state_off + e] : T(0));
  }
}

// ---------------------------------------------------------------------------
// Tiled leap-frog step for 2D/3D acoustics.  A block of 32 x 8 threads owns a
// 32 x 32 x-y tile of one z plane (4 rows per thread).  It stages the current level's
// p, u, v over the tile plus an R-wide periodic halo in shared memory with coalesced
// loads, takes the x- and y-stencils from there, and the z-stencils (3D) through the
// cache.  Same arithmetic and the same last-step averaging/combine as k_lf.
// ---------------------------------------------------------------------------

__device__ __forceinline__ int wrap_any(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

// Tile staging: the (kTileX + 2R) x (kTileY + 2R) points of a tile and its halo are spread over
// the 256 threads of a block, iteration it of thread t taking point t + 256 it (row r, column cl
// of the staged tile).  Kernels run the iterations in fully unrolled loops that issue all of a
// thread's loads before its shared-memory stores, so that they are in flight together.
template <int R>
struct TileStage {
  static constexpr int W = kTileX + 2 * R, Hh = kTileY + 2 * R, NE = W * Hh, NIT = (NE + 255) / 256;
  // row and column of iteration it, false past the tile
  static __device__ __forceinline__ bool rc(int it, int& r, int& cl) {
    const int e = threadIdx.y * kTileX + threadIdx.x + 256 * it;
    if (e >= NE) return false;
    r = e / W;
    cl = e - r * W;
    return true;
  }
  // point offset (periodic) of staged row r, column cl, within z plane `plane`
  static __device__ __forceinline__ int64_t at(int r, int cl, int x0, int y0, int nx, int ny, int64_t plane) {
    int gy = y0 - R + r;
    if (gy < 0 || gy >= ny) gy = wrap_any(gy, ny);
    int gx = x0 - R + cl;
    if (gx < 0 || gx >= nx) gx = wrap_any(gx, nx);
    return plane + (int64_t)gy * nx + gx;
  }
  // the same as a 32-bit offset (a problem has fewer than 2^31 points per field)
  static __device__ __forceinline__ int at32(int r, int cl, int x0, int y0, int nx, int ny, int plane) {
    int gy = y0 - R + r;
    if (gy < 0 || gy >= ny) gy = wrap_any(gy, ny);
    int gx = x0 - R + cl;
    if (gx < 0 || gx >= nx) gx = wrap_any(gx, nx);
    return plane + gy * nx + gx;
  }
};

// 16-byte vector of a state type (4 floats, 2 doubles, 2 FP32 pairs)
template <class T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
};
template <>
struct Vec16<double> {
  using type = double2;
};
template <>
struct Vec16<dsf> {
  using type = float4;
};

// resident blocks per SM the register budget of k_lf_tiled aims at, each measured best against
// its neighbours: FP32 2D 5, FP32 3D 4 (one fewer than before the increment form, whose f0 and
// scaled-media operands take registers); 8-byte states 3 in 2D and 2 in 3D.  The FP32 values can
// be set at build time for such measurements.
#ifndef GBS_LF_BLOCKS_F32_2D
#define GBS_LF_BLOCKS_F32_2D 5
#endif
#ifndef GBS_LF_BLOCKS_F32_3D
#define GBS_LF_BLOCKS_F32_3D 4
#endif
template <typename T, int DIM, int R>
constexpr int lf_min_blocks() {
  return sizeof(T) == 4 ? (DIM == 2 ? GBS_LF_BLOCKS_F32_2D : GBS_LF_BLOCKS_F32_3D) : (DIM == 2 ? 3 : 2);
}

// TMA staging helpers (inline PTX): shared-window address, mbarrier, 4D tensor copy
__device__ __forceinline__ unsigned smem_u32(const void* ptr) {
  return static_cast<unsigned>(__cvta_generic_to_shared(ptr));
}
constexpr long long kTmaSpin = 1ll << 22;   // try_wait polls before a copy counts as lost

// First and last sequence to finish among the slot's scheduled sequences when all of them
// advance level by level together (a sequence-fused step): by step count, ties in index order.
__device__ __forceinline__ void seq_first_last_by_steps(const StepPlan& p, const SlotDev& s, int k, bool& first,
                                                        bool& last) {
  const unsigned msk = p.seq_mask & ((1u << s.m) - 1u);
  const int N = s.steps[k];
  first = true;
  last = !p.partial;
  for (int i = 0; i < s.m; ++i) {
    if (!((msk >> i) & 1u) || i == k) continue;
    if (s.steps[i] < N || (s.steps[i] == N && i < k)) first = false;
    if (s.steps[i] > N || (s.steps[i] == N && i > k)) last = false;
  }
}

// kMulti: the sequence-fused variant (several sequences per launch, own level pairs), given one
// resident block per SM less for the registers its loop over the sequences keeps live
// staging tile of k_lf_tiled: HX columns on each side of the tile (>= R and a whole number of
// 16-byte vectors), R rows above and below
template <typename T, int R>
struct LfTile {
  static constexpr int Hh = kTileY + 2 * R, HX = 4, WS = kTileX + 2 * HX;
  using Arr = T[3][Hh][WS];
};

// Problem of a tiled-grid block (binary search over the tiled-grid offsets).
__device__ __forceinline__ int tiled_problem(const StepPlan& p, int64_t blk) {
  int lo = 0, hi = p.batch - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.probs[mid].tblk_begin <= blk) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// One leap-frog level n of sequence k over one tile (the body of k_lf_tiled): stage the tile of
// y_n, then update each of the thread's rows.  `uses` counts the earlier copies on tma_bar in
// this block (0: the barrier is initialised here).  Returns false when a tensor copy did not
// complete in time (GBS_ERR_TIMEOUT latched; the block must stop).
template <typename T, int DIM, int R, bool kVec, bool kTma>
__device__ __forceinline__ bool lf_tile_level(const StepPlan& p, const T* y_in, typename out_of<T>::type* y_out,
                                              int k, int n, const CUtensorMap& tmap, const SeqLevels& lv,
                                              typename LfTile<T, R>::Arr& sh, unsigned long long& tma_bar,
                                              int uses, int lo, int64_t blk) {
  constexpr int Hh = LfTile<T, R>::Hh, HX = LfTile<T, R>::HX, WS = LfTile<T, R>::WS;
  const ProbDev& q = p.probs[lo];
  const SlotDev& s = p.slots[q.slot];
  if (k >= s.m) return true;
  const int N = s.steps[k];
  if (n > N) return true;
  const int tile = (int)(blk - q.tblk_begin);
  const int tx = tile % q.tiles_x;
  const int rest = tile / q.tiles_x;
  const int ty = rest % q.tiles_y;
  const int z = rest / q.tiles_y;
  const int nx = q.n[0], ny = q.n[1], nz = q.n[2];
  const int x0 = tx * kTileX, y0 = ty * kTileY;
  const int64_t P = q.pts;
  // 3D: offsets within one field (fewer than 2^31 points per field, checked at creation) are
  // 32-bit and every field has its own base pointer; 2D: 64-bit element offsets, which need
  // fewer registers (each measured faster for its case)
  using Off = typename std::conditional<DIM == 3, int, int64_t>::type;
  const Off plane = (Off)z * nx * ny;
  T h, h2;
  step_sizes(p, lo, k, h, h2);
  // level buffers: the handle's pair, or sequence k's own pair in a sequence-fused step
  T* const L0 = (lv.base ? static_cast<T*>(lv.base) + (2 * k) * lv.stride : static_cast<T*>(p.L0)) + q.state_off;
  T* const L1 = (lv.base ? static_cast<T*>(lv.base) + (2 * k + 1) * lv.stride : static_cast<T*>(p.L1)) + q.state_off;
  const T* cur = (n & 1) ? L1 : L0;
  T* dst = (n & 1) ? L0 : L1;                          // y_(n+1) overwrites y_(n-1)
  const T* prev = (n == 1) ? (y_in + q.state_off) : dst;
  constexpr int F = 1 + DIM;
  const T* kap = static_cast<const T*>(p.kappa) + q.media_off;
  const T* bmed = static_cast<const T*>(p.b) + q.media_off;
  const int x = x0 + threadIdx.x;
  const Off o0 = plane + (Off)(y0 + (int)threadIdx.y) * nx + x;   // this thread's point in row 0
  // z-neighbour plane offsets (3D, periodic)
  int dzp[R], dzm[R];
#pragma unroll
  for (int j = 1; j <= R; ++j) {
    const int zp = z + j >= nz ? z + j - nz : z + j;
    const int zm = z - j < 0 ? z - j + nz : z - j;
    dzp[j - 1] = (zp - z) * nx * ny;
    dzm[j - 1] = (zm - z) * nx * ny;
  }
  // FP32: increment form (gbs_stencil.cuh), d_(n+1) = d_(n-1) + 2h f0 + 2h A d_n, d_0 = 0
  constexpr bool kInc = std::is_same<T, float>::value;
  const T* f0v = static_cast<const T*>(p.f0) + q.state_off;
  float gh = 0.f, gl = 0.f, sch = 0.f, scl = 0.f;
  if constexpr (kInc) {
    // the forcing's 2h, and -2h / (div dx_0) for the integer-weight stencil sums, as float pairs
    const float4 hq = p.hkq[lo * GBS_MAX_SEQ + k];
    gh = hq.x;
    gl = hq.y;
    sch = -hq.z;
    scl = -hq.w;
  }
  const bool prev_zero = kInc && n == 1;
  // point-wise operands of a row (previous level, media, f0 in the increment form, and in 3D
  // the z-neighbours of p and w), loaded one row ahead of their use; the first row's before the
  // tile barrier
  T nprev[F], nf0[F], nkv = T(0), nbv = T(0), nzp[R][2], nzm[R][2];
  auto fetch_row = [&](int i) {
    const int y = y0 + threadIdx.y + 8 * i;
    if (x >= nx || y >= ny) return;
    const Off o = o0 + (Off)(8 * i) * nx;
#pragma unroll
    for (int fl = 0; fl < F; ++fl) {
      nprev[fl] = prev_zero ? T(0) : DIM == 3 ? (prev + fl * P)[o] : prev[fl * P + o];
      if constexpr (kInc) nf0[fl] = DIM == 3 ? ldg(f0v + fl * P + o) : ldg(f0v + (fl * P + o));
    }
    nkv = ldg(kap + o);
    nbv = ldg(bmed + o);
    if (DIM == 3) {
#pragma unroll
      for (int j = 0; j < R; ++j) {
        nzp[j][0] = ldg(cur + (o + dzp[j]));
        nzp[j][1] = ldg(cur + 3 * P + (o + dzp[j]));
        nzm[j][0] = ldg(cur + (o + dzm[j]));
        nzm[j][1] = ldg(cur + 3 * P + (o + dzm[j]));
      }
    }
  };
  // stage p, u, v of the current level (tile + halo, periodic) with all of a thread's loads issued
  // before its shared stores; the first row's point-wise operands are fetched in between.  kVec
  // (every problem's nx a multiple of 4, so every row and every problem offset is a whole number
  // of 16-byte vectors; the tile's columns start at multiples of 32 and HX is whole vectors, so
  // every vector stays inside one period): the WS staged columns move as 16-byte vectors; else
  // the tile's W = kTileX + 2 R columns move point by point.
  constexpr int VW = 16 / sizeof(T);
  using V = typename Vec16<T>::type;
  auto stage_vectors = [&]() {
    constexpr int GR = WS / VW, NV = Hh * GR, NITV = (NV + 255) / 256;
    const int ltid = threadIdx.y * kTileX + threadIdx.x;
    V vs[3][NITV];
#pragma unroll
    for (int it = 0; it < NITV; ++it) {
      const int e = ltid + 256 * it;
      if (e < NV) {
        const int r = e / GR, g = e - r * GR;
        int gy = y0 - R + r;
        if (gy < 0 || gy >= ny) gy = wrap_any(gy, ny);
        int gx = x0 - HX + g * VW;
        if (gx < 0 || gx >= nx) gx = wrap_any(gx, nx);
        const Off o = plane + (Off)gy * nx + gx;
#pragma unroll
        for (int f = 0; f < 3; ++f) vs[f][it] = __ldg(reinterpret_cast<const V*>(cur + f * P + o));
      }
    }
    fetch_row(0);
#pragma unroll
    for (int it = 0; it < NITV; ++it) {
      const int e = ltid + 256 * it;
      if (e < NV) {
        const int r = e / GR, g = e - r * GR;
#pragma unroll
        for (int f = 0; f < 3; ++f) *reinterpret_cast<V*>(&sh[f][r][g * VW]) = vs[f][it];
      }
    }
  };
  if constexpr (kTma) {
    // Tensor-memory-access staging (every nx a multiple of 4, a single FP32 problem): when the
    // tile's box of WS columns x Hh rows lies inside the grid, thread (0, 0) starts one 4D copy
    // of p, u, v (coordinates x0 - HX, a multiple of 4 floats, y0 - R, z, field 0) that
    // completes on an mbarrier, while every thread fetches its first row's point-wise operands;
    // boxes that cross the periodic edge use the vector loads.  A copy that does not complete
    // within kTmaSpin polls latches GBS_ERR_TIMEOUT and the block returns.
    const bool inside = x0 >= HX && x0 + kTileX + HX <= nx && y0 >= R && y0 + kTileY + R <= ny;
    if (inside) {
      const unsigned bar = smem_u32(&tma_bar);
      const bool lead = threadIdx.x == 0 && threadIdx.y == 0;
      if (uses == 0) {
        if (lead) {
          asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
          asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        __syncthreads();
      } else if (lead) {   // the tile's earlier reads (ordered by the caller's barrier) before the copy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      }
      if (lead) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"((unsigned)sizeof(sh))
                     : "memory");
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(&sh[0][0][0])),
            "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(x0 - HX), "r"(y0 - R), "r"(z),
            "r"(lv.base ? (2 * k + (n & 1)) * F : 0), "r"(bar)
            : "memory");
      }
      fetch_row(0);
      unsigned ready = 0;
      for (long long it = 0; it < kTmaSpin && !ready; ++it)
        asm volatile(
            "{\n\t.reg .pred P;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, P;\n\t}"
            : "=r"(ready)
            : "r"(bar), "r"((unsigned)(uses & 1))
            : "memory");
      if (__syncthreads_or(!ready)) {
        if (lead) atomicCAS(p.err, 0, (int)GBS_ERR_TIMEOUT);
        return false;
      }
    } else {
      stage_vectors();
    }
  } else if constexpr (kVec) {
    stage_vectors();
  } else {
    using TS = TileStage<R>;
    T stg[3][TS::NIT];
#pragma unroll
    for (int it = 0; it < TS::NIT; ++it) {
      int r, cl;
      if (TS::rc(it, r, cl)) {
        Off o;
        if constexpr (DIM == 3) o = TS::at32(r, cl, x0, y0, nx, ny, plane);
        else o = TS::at(r, cl, x0, y0, nx, ny, plane);
        stg[0][it] = ldg(cur + o);
        stg[1][it] = ldg(cur + P + o);
        stg[2][it] = ldg(cur + 2 * P + o);
      }
    }
    fetch_row(0);
#pragma unroll
    for (int it = 0; it < TS::NIT; ++it) {
      int r, cl;
      if (TS::rc(it, r, cl)) {
        sh[0][r][cl + HX - R] = stg[0][it];
        sh[1][r][cl + HX - R] = stg[1][it];
        sh[2][r][cl + HX - R] = stg[2][it];
      }
    }
  }
  __syncthreads();
  // FP32 (integer-weight form): idx unused, idy and idz the spacing ratios dx_0 / dx_d
  const T idx = T(q.inv_dx[0]);
  const T idy = kInc ? T(q.rr[1]) : T(q.inv_dx[1]);
  const T idz = kInc ? T(q.rr[2]) : T(q.inv_dx[2]);
  if (x >= nx) return true;
  const double c = s.c[k];
  bool first, last;
  if (lv.base) seq_first_last_by_steps(p, s, k, first, last);
  else seq_first_last(p, k, s.m, first, last);
#pragma unroll
  for (int i = 0; i < kTileRows; ++i) {
    const int ly = threadIdx.y + 8 * i;
    const int y = y0 + ly;
    if (y >= ny) break;
    T pv[F], pg[F], zpv[R][2], zmv[R][2];
#pragma unroll
    for (int fl = 0; fl < F; ++fl) {
      pv[fl] = nprev[fl];
      if constexpr (kInc) pg[fl] = pv[fl] + mul_split(gh, gl, nf0[fl]);
      else pg[fl] = pv[fl];
    }
    const T kv = nkv, bv = nbv;
    if (DIM == 3) {
#pragma unroll
      for (int j = 0; j < R; ++j) {
        zpv[j][0] = nzp[j][0];
        zpv[j][1] = nzp[j][1];
        zmv[j][0] = nzm[j][0];
        zmv[j][1] = nzm[j][1];
      }
    }
    if (i + 1 < kTileRows) fetch_row(i + 1);
    const int r = ly + R, cc = threadIdx.x + HX;
    // stencil sums: FP32 states with the integer weights (times div), otherwise the weights
    T sxu = T(0), sxp = T(0), syv = T(0), syp = T(0);
#pragma unroll
    for (int j = 1; j <= R; ++j) {
      const T a = kInc ? T(fd_int<R>(j)) : T(fd_coef<R>(j));
      sxp += a * (sh[0][r][cc + j] - sh[0][r][cc - j]);
      sxu += a * (sh[1][r][cc + j] - sh[1][r][cc - j]);
      syp += a * (sh[0][r + j][cc] - sh[0][r - j][cc]);
      syv += a * (sh[2][r + j][cc] - sh[2][r - j][cc]);
    }
    const Off o = o0 + (Off)(8 * i) * nx;
    T szp = T(0), szw = T(0);
    if (DIM == 3) {
#pragma unroll
      for (int j = 1; j <= R; ++j) {
        const T a = kInc ? T(fd_int<R>(j)) : T(fd_coef<R>(j));
        szp += a * (zpv[j - 1][0] - zmv[j - 1][0]);
        szw += a * (zpv[j - 1][1] - zmv[j - 1][1]);
      }
    }
    T f[kMaxFields];
    // FP32: the scaled media s kappa and s b (s = -2h / (div dx_0)) as float pairs, the rounded
    // product plus its exact error and the lo part
    float kh = 0.f, kl = 0.f, bh = 0.f, bl = 0.f;
    if constexpr (kInc) {
      // the stencil sums of div dx_0 f(d_n) without the media; idy, idz are dx_0 / dx_d here
      T sd = fmaf(idy, syv, sxu);
      if (DIM == 3) sd = fmaf(idz, szw, sd);
      f[0] = sd;
      f[1] = sxp;
      f[2] = idy * syp;
      if (DIM == 3) f[3] = idz * szp;
      kh = __fmul_rn(sch, kv);
      kl = fmaf(scl, kv, fmaf(sch, kv, -kh));
      bh = __fmul_rn(sch, bv);
      bl = fmaf(scl, bv, fmaf(sch, bv, -bh));
    } else {
      T div = sxu * idx + syv * idy;
      if (DIM == 3) div += szw * idz;
      f[0] = -kv * div;
      f[1] = -bv * (sxp * idx);
      f[2] = -bv * (syp * idy);
      if (DIM == 3) f[3] = -bv * (szp * idz);
    }
    // prev + 2h f (FP32: the pair-scaled media times the stencil sums)
    auto lf_update = [&](int fl, T pv_, T fv) -> T {
      if constexpr (kInc) {
        const float mh = fl == 0 ? kh : bh, ml = fl == 0 ? kl : bl;
        return fmaf(mh, fv, fmaf(ml, fv, pv_));
      } else {
        return pv_ + h2 * fv;
      }
    };
    if (n < N) {
#pragma unroll
      for (int fl = 0; fl < F; ++fl) {
        if (DIM == 3) (dst + fl * P)[o] = lf_update(fl, pg[fl], f[fl]);
        else dst[fl * P + o] = lf_update(fl, pg[fl], f[fl]);
      }
    } else {
      double* acc = p.acc + q.state_off;
      auto* yo = y_out + q.state_off;
#pragma unroll
      for (int fl = 0; fl < F; ++fl) {
        const int64_t e = fl * P + o;
        const T yc = fl == 0 ? sh[0][r][cc] : fl == 1 ? sh[1][r][cc] : fl == 2 ? sh[2][r][cc] : ldg(cur + e);
        const T yp = lf_update(fl, pg[fl], f[fl]);
        combine_last<T, typename out_of<T>::type, DIM == 3>(acc, e, first, last, c, gragg_avg(pv[fl], yc, yp), yo,
                     kInc && first && !p.partial ? y_in[q.state_off + e] : T(0));
      }
    }
  }
  return true;
}

template <typename T, int DIM, int R, bool kVec, bool kTma>
__global__ void __launch_bounds__(256, lf_min_blocks<T, DIM, R>())
    k_lf_tiled(const StepPlan p, const T* y_in, typename out_of<T>::type* y_out, int k, int n,
               const __grid_constant__ CUtensorMap tmap) {
  // 128-byte aligned: the tensor copy's destination (its box is [3][Hh][WS], x fastest)
  __shared__ __align__(128) typename LfTile<T, R>::Arr sh;
  __shared__ __align__(8) unsigned long long tma_bar;
  const int64_t blk = blockIdx.x;
  lf_tile_level<T, DIM, R, kVec, kTma>(p, y_in, y_out, k, n, tmap, SeqLevels{nullptr, 0, nullptr}, sh, tma_bar, 0,
                                       tiled_problem(p, blk), blk);
}

// The sequence-fused step: level n of every sequence of kmask (na of them), each from its own
// level pair (lv), one block per tile and sequence with the sequence index running fastest, so
// that the na blocks of a tile run side by side and their reads of the tile's f0 and media after
// the first are served by the cache.  At most one scheduled sequence finishes at level n (step
// counts are distinct), so the blocks' combine updates never meet.
template <typename T, int DIM, int R, bool kVec, bool kTma>
__global__ void __launch_bounds__(256, lf_min_blocks<T, DIM, R>())
    k_lf_tiled_seqs(const StepPlan p, const T* y_in, typename out_of<T>::type* y_out, uint32_t kmask, int na, int n,
                    const __grid_constant__ CUtensorMap tmap, const SeqLevels lv) {
  __shared__ __align__(128) typename LfTile<T, R>::Arr sh;
  __shared__ __align__(8) unsigned long long tma_bar;
  const int64_t blk = blockIdx.x / na;
  uint32_t km = kmask;
  for (int i = blockIdx.x % na; i > 0; --i) km &= km - 1;   // the (blockIdx.x mod na)-th sequence
  lf_tile_level<T, DIM, R, kVec, kTma>(p, y_in, y_out, __ffs(km) - 1, n, tmap, lv, sh, tma_bar, 0,
                                       tiled_problem(p, blk), blk);
}

// Tiled leap-frog step for 2D/3D acoustics in FP32 pairs (GBS_F32X2), two pair values per
// packed instruction: the x-stencils of (p, u) and the y-stencils of (p, v) run lane by lane
// on f32x2 (ds2), as integer-weight sums (isum_x2) whose divisor is folded into 2h.  The tile
// holds (p.hi, u.hi, p.lo, u.lo) and (p.hi, v.hi, p.lo, v.lo) per point so that each stencil
// operand is one 16-byte shared load.  Same steps, averaging and FP64 combine as k_lf_tiled.
template <int DIM, int R, bool kVec>
__global__ void __launch_bounds__(256, DIM == 3 ? 3 : 4) k_lf_tiled_x2(const StepPlan p, const dsf* y_in, double* y_out, int k, int n) {
  // staged columns: HX = 4 on each side of the tile (>= R, whole 16-byte vectors of two pairs)
  constexpr int Hh = kTileY + 2 * R, HX = 4, WS = kTileX + 2 * HX;
  __shared__ float4 spu[Hh][WS];   // (p.hi, u.hi, p.lo, u.lo)
  __shared__ float4 spv[Hh][WS];   // (p.hi, v.hi, p.lo, v.lo)
  int lo = 0, hi = p.batch - 1;
  const int64_t blk = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.probs[mid].tblk_begin <= blk) lo = mid;
    else hi = mid - 1;
  }
  const ProbDev& q = p.probs[lo];
  const SlotDev& s = p.slots[q.slot];
  if (k >= s.m) return;
  const int N = s.steps[k];
  if (n > N) return;
  const int tile = (int)(blk - q.tblk_begin);
  const int tx = tile % q.tiles_x;
  const int rest = tile / q.tiles_x;
  const int ty = rest % q.tiles_y;
  const int z = rest / q.tiles_y;
  const int nx = q.n[0], ny = q.n[1], nz = q.n[2];
  const int x0 = tx * kTileX, y0 = ty * kTileY;
  const int64_t P = q.pts;
  const int64_t plane = (int64_t)z * nx * ny;
  dsf h, h2;
  step_sizes(p, lo, k, h, h2);
  h2 = h2 * dsf(1.0 / fd_div<R>());   // the stencil sums below carry the integer weights' divisor
  dsf* const L0 = static_cast<dsf*>(p.L0) + q.state_off;
  dsf* const L1 = static_cast<dsf*>(p.L1) + q.state_off;
  const dsf* cur = (n & 1) ? L1 : L0;
  dsf* dst = (n & 1) ? L0 : L1;
  const dsf* prev = (n == 1) ? (y_in + q.state_off) : dst;
  const dsf* kap = static_cast<const dsf*>(p.kappa) + q.media_off;
  const dsf* bmed = static_cast<const dsf*>(p.b) + q.media_off;
  const int x = x0 + threadIdx.x;
  // point-wise operands of a row (previous level, media), loaded one row ahead of their use;
  // the first row's before the tile barrier
  dsf nprev[4], nkv, nbv;
  auto fetch_row = [&](int i) {
    const int y = y0 + threadIdx.y + 8 * i;
    if (x >= nx || y >= ny) return;
    const int64_t pt = plane + (int64_t)y * nx + x;
#pragma unroll
    for (int fl = 0; fl < 1 + DIM; ++fl) nprev[fl] = ldg(prev + fl * P + pt);
    nkv = ldg(kap + pt);
    nbv = ldg(bmed + pt);
  };
  // stage the tile and its halo with all of a thread's loads issued before its shared stores (the
  // first row's point-wise operands in between): as 16-byte vectors of two pairs when kVec
  // (every nx a multiple of 4, the staged rows widened to WS columns), else point by point
  if constexpr (kVec) {
    constexpr int GR = WS / 2, NV = Hh * GR, NITV = (NV + 255) / 256;
    const int ltid = threadIdx.y * kTileX + threadIdx.x;
    float4 vs[3][NITV];   // (hi, lo) of two consecutive points of p, u, v
#pragma unroll
    for (int it = 0; it < NITV; ++it) {
      const int e = ltid + 256 * it;
      if (e < NV) {
        const int r = e / GR, g = e - r * GR;
        int gy = y0 - R + r;
        if (gy < 0 || gy >= ny) gy = wrap_any(gy, ny);
        int gx = x0 - HX + 2 * g;
        if (gx < 0 || gx >= nx) gx = wrap_any(gx, nx);
        const dsf* a = cur + plane + (int64_t)gy * nx + gx;
#pragma unroll
        for (int f = 0; f < 3; ++f) vs[f][it] = __ldg(reinterpret_cast<const float4*>(a + f * P));
      }
    }
    fetch_row(0);
#pragma unroll
    for (int it = 0; it < NITV; ++it) {
      const int e = ltid + 256 * it;
      if (e < NV) {
        const int r = e / GR, g = e - r * GR;
        const float4 pp = vs[0][it], uu = vs[1][it], vv = vs[2][it];
        spu[r][2 * g] = make_float4(pp.x, uu.x, pp.y, uu.y);
        spu[r][2 * g + 1] = make_float4(pp.z, uu.z, pp.w, uu.w);
        spv[r][2 * g] = make_float4(pp.x, vv.x, pp.y, vv.y);
        spv[r][2 * g + 1] = make_float4(pp.z, vv.z, pp.w, vv.w);
      }
    }
  } else {
    using TS = TileStage<R>;
    dsf stg[3][TS::NIT];
#pragma unroll
    for (int it = 0; it < TS::NIT; ++it) {
      int r, cl;
      if (TS::rc(it, r, cl)) {
        const dsf* a = cur + TS::at(r, cl, x0, y0, nx, ny, plane);
        stg[0][it] = ldg(a);
        stg[1][it] = ldg(a + P);
        stg[2][it] = ldg(a + 2 * P);
      }
    }
    fetch_row(0);
#pragma unroll
    for (int it = 0; it < TS::NIT; ++it) {
      int r, cl;
      if (TS::rc(it, r, cl)) {
        const dsf pp = stg[0][it], uu = stg[1][it], vv = stg[2][it];
        spu[r][cl + HX - R] = make_float4(pp.hi, uu.hi, pp.lo, uu.lo);
        spv[r][cl + HX - R] = make_float4(pp.hi, vv.hi, pp.lo, vv.lo);
      }
    }
  }
  __syncthreads();
  const bool unit = q.inv_dx[0] == 1.0 && q.inv_dx[1] == 1.0 && (DIM < 3 || q.inv_dx[2] == 1.0);
  const dsf idx = dsf(q.inv_dx[0]), idy = dsf(q.inv_dx[1]), idz = dsf(q.inv_dx[2]);
  if (x >= nx) return;
  const double c = s.c[k];
  bool first, last;
  seq_first_last(p, k, s.m, first, last);
#pragma unroll
  for (int i = 0; i < kTileRows; ++i) {
    const int ly = threadIdx.y + 8 * i;
    const int y = y0 + ly;
    if (y >= ny) break;
    const int r = ly + R, cc = threadIdx.x + HX;
    dsf pv[4];
#pragma unroll
    for (int fl = 0; fl < 4; ++fl) pv[fl] = nprev[fl];
    const dsf kv = nkv, bv = nbv;
    if (i + 1 < kTileRows) fetch_row(i + 1);
    // (D_x p, D_x u) and (D_y p, D_y v) times the integer weights' divisor, unscaled by dx
    ds2 sx = isum_x2<R>([&](int j) { const float4 v = spu[r][cc + j]; return make_float2(v.x, v.y); },
                        [&](int j) { const float4 v = spu[r][cc + j]; return make_float2(v.z, v.w); });
    ds2 sy = isum_x2<R>([&](int j) { const float4 v = spv[r + j][cc]; return make_float2(v.x, v.y); },
                        [&](int j) { const float4 v = spv[r + j][cc]; return make_float2(v.z, v.w); });
    const int64_t pt = plane + (int64_t)y * nx + x;
    ds2 sz{};                                    // (D_z p, D_z w) times the divisor, 3D only
    if (DIM == 3) {
      ds2 zv[2 * R + 1];                         // (p, w) at z - R .. z + R (the centre unused)
#pragma unroll
      for (int j = 1; j <= R; ++j) {
        const int zp = z + j >= nz ? z + j - nz : z + j;
        const int zm = z - j < 0 ? z - j + nz : z - j;
        const int64_t op = (int64_t)(zp - z) * nx * ny, om = (int64_t)(zm - z) * nx * ny;
        zv[R + j] = make_ds2(ldg(cur + pt + op), ldg(cur + 3 * P + pt + op));
        zv[R - j] = make_ds2(ldg(cur + pt + om), ldg(cur + 3 * P + pt + om));
      }
      sz = isum_x2<R>([&](int j) { return zv[R + j].hi; }, [&](int j) { return zv[R + j].lo; });
    }
    if (!unit) {
      sx = ds2_mul(sx, idx.hi, idx.lo);
      sy = ds2_mul(sy, idy.hi, idy.lo);
      if (DIM == 3) sz = ds2_mul(sz, idz.hi, idz.lo);
    }
    dsf div = lane_y(sx) + lane_y(sy);
    if (DIM == 3) div += lane_y(sz);
    const dsf fp = -(kv * div);
    const ds2 fuv = ds2_mul(make_ds2(lane_x(sx), lane_x(sy)), make_ds2(-bv, -bv));   // (f_u, f_v)
    dsf fw = dsf(0);
    if (DIM == 3) fw = -(bv * lane_x(sz));
    if (n < N) {
      dst[pt] = pv[0] + h2 * fp;
      const ds2 nuv = make_ds2(pv[1], pv[2]) + ds2_mul(fuv, h2.hi, h2.lo);
      dst[P + pt] = lane_x(nuv);
      dst[2 * P + pt] = lane_y(nuv);
      if (DIM == 3) dst[3 * P + pt] = pv[3] + h2 * fw;
    } else {
      double* acc = p.acc + q.state_off;
      double* yo = y_out + q.state_off;
      const float4 a = spu[r][cc], b = spv[r][cc];
      const dsf cur_f[4] = {dsf(a.x, a.z), dsf(a.y, a.w), dsf(b.y, b.w), DIM == 3 ? ldg(cur + 3 * P + pt) : dsf(0)};
      const dsf f[4] = {fp, lane_x(fuv), lane_y(fuv), fw};
#pragma unroll
      for (int fl = 0; fl < 1 + DIM; ++fl) {
        const int64_t e = fl * P + pt;
        const dsf ym = pv[fl];
        const dsf yp = ym + h2 * f[fl];
        const double ys = (double)gragg_avg(ym, cur_f[fl], yp);
        const double a2 = first ? c * ys : fma(c, ys, acc[e]);
        if (last) yo[e] = a2;
        else acc[e] = a2;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Adjoint kernels (acoustics)
// ---------------------------------------------------------------------------

// Forward level store: lev[n+1] = lev[n-1] + 2h f(lev[n]) (n >= 1), lev[1] = y_in + h f0.
template <typename T, int DIM, int R>
__global__ void __launch_bounds__(kPlainBlock) k_adj_fwd(const StepPlan p, const T* __restrict__ y_in,
                                                         T* lev, int64_t lev_stride, int k, int n) {
  const Loc L = locate(p);
  if (L.prob < 0) return;
  const ProbDev& q = p.probs[L.prob];
  const SlotDev& s = p.slots[q.slot];
  if (k >= s.m) return;
  const int N = s.steps[k];
  if (n > N) return;
  constexpr int F = 1 + DIM;
  const double hd = p.hk[L.prob * GBS_MAX_SEQ + k];
  const T* y0 = y_in + q.state_off;
  auto level = [&](int j) -> T* { return lev + (int64_t)j * lev_stride + q.state_off; };
  if (n == 0) {
    const T h = T(hd);
    const T* f0 = static_cast<const T*>(p.f0) + q.state_off;
    T* d = level(1);
#pragma unroll
    for (int fl = 0; fl < F; ++fl) {
      const int64_t e = fl * q.pts + L.i;
      d[e] = y0[e] + h * f0[e];
    }
    return;
  }
  const T* cur = level(n);
  const T* prev = (n == 1) ? y0 : level(n - 1);
  T* dst = level(n + 1);
  const PointGeo g = geo_of(q, L.i);
  T inv_dx[3];
  load_inv_dx(q, inv_dx);
  const T kap = ldg(static_cast<const T*>(p.kappa) + q.media_off + L.i);
  const T bb = ldg(static_cast<const T*>(p.b) + q.media_off + L.i);
  T f[kMaxFields];
  rhs_point<T, SYS_ACOUSTIC, DIM, R>(cur, q.pts, g, inv_dx, kap, bb, f);
  const T h2 = T(2.0 * hd);
#pragma unroll
  for (int fl = 0; fl < F; ++fl) {
    const int64_t e = fl * q.pts + L.i;
    dst[e] = prev[e] + h2 * f[fl];
  }
}

// Reverse step j (N >= j >= 1), in place over the buffer of M[j+2]:
//   M[j] = M[j+2] + init_j + 2h A^T M[j+1],  init_N = w/2, init_(N-1) = w/4 (w = c_k lam_out),
//   M[N+2] = 0;  g += 2h mu_p (-div y_j) with mu = M[j+1].
// j == N + 1 initialises M[N+1] = w/4.
template <typename T, int DIM, int R>
__global__ void __launch_bounds__(kPlainBlock) k_adj_rev(const StepPlan p, const T* __restrict__ y_in,
                                                         const T* __restrict__ lev, int64_t lev_stride,
                                                         const T* __restrict__ lam_out, T* mA, T* mB,
                                                         double* grad, int k, int jrev) {
  const Loc L = locate(p);
  if (L.prob < 0) return;
  const ProbDev& q = p.probs[L.prob];
  const SlotDev& s = p.slots[q.slot];
  if (k >= s.m) return;
  const int N = s.steps[k];
  // jrev counts launches 0.. ; launch t handles j = N + 1 - t (problems with smaller N skip)
  const int j = N + 1 - jrev;
  if (j < 1) return;
  constexpr int F = 1 + DIM;
  const double hd = p.hk[L.prob * GBS_MAX_SEQ + k];
  const double c = s.c[k];
  // M[j] lives in buffer ((N + 1 - j) & 1) == 0 ? A : B
  T* dst = (((N + 1 - j) & 1) == 0 ? mA : mB) + q.state_off;
  const T* src = (((N + 1 - j) & 1) == 0 ? mB : mA) + q.state_off;  // M[j+1]
  const T* lo = lam_out + q.state_off;
  if (j == N + 1) {
#pragma unroll
    for (int fl = 0; fl < F; ++fl) {
      const int64_t e = fl * q.pts + L.i;
      dst[e] = T(0.25 * c * (double)lo[e]);
    }
    return;
  }
  const PointGeo g = geo_of(q, L.i);
  T inv_dx[3];
  load_inv_dx(q, inv_dx);
  const T* kappa = static_cast<const T*>(p.kappa) + q.media_off;
  const T* bmed = static_cast<const T*>(p.b) + q.media_off;
  T at[kMaxFields];
  rhs_T_point<T, DIM, R>(src, q.pts, g, inv_dx, kappa, bmed, at);
  const T h2 = T(2.0 * hd);
#pragma unroll
  for (int fl = 0; fl < F; ++fl) {
    const int64_t e = fl * q.pts + L.i;
    T base = (j <= N - 1) ? dst[e] : T(0);          // M[j+2]
    if (j == N) base += T(0.5 * c * (double)lo[e]);
    if (j == N - 1) base += T(0.25 * c * (double)lo[e]);
    dst[e] = base + h2 * at[fl];
  }
  // gradient term 2h mu_p (-div y_j), y_j = level j (y_in for j == 0, never here)
  const T* yj = lev + (int64_t)j * lev_stride + q.state_off;
  const T dv = div_point<T, DIM, R>(yj, q.pts, g, inv_dx);
  grad[q.media_off + L.i] += 2.0 * hd * (double)src[L.i] * (-(double)dv);
}

// ---------------------------------------------------------------------------
// Tiled adjoint kernels for 2D/3D acoustics: the same tiles as k_lf_tiled (32 x 32 x-y tiles
// of one z plane, 32 x 8 threads, 4 rows each, periodic halo staged in shared memory).
// ---------------------------------------------------------------------------

struct TileLoc {
  int prob, tx, ty, z;
};

__device__ __forceinline__ TileLoc tile_of(const StepPlan& p) {
  int lo = 0, hi = p.batch - 1;
  const int64_t blk = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.probs[mid].tblk_begin <= blk) lo = mid;
    else hi = mid - 1;
  }
  const ProbDev& q = p.probs[lo];
  const int tile = (int)(blk - q.tblk_begin);
  TileLoc t;
  t.prob = lo;
  t.tx = tile % q.tiles_x;
  const int rest = tile / q.tiles_x;
  t.ty = rest % q.tiles_y;
  t.z = rest / q.tiles_y;
  return t;
}

// Forward level store, tiled: lev[n+1] = lev[n-1] + 2h f(lev[n]) (n >= 1), lev[1] = y_in + h f0.
template <typename T, int DIM, int R, bool kVec>
__global__ void __launch_bounds__(256) k_adj_fwd_tiled(const StepPlan p, const T* __restrict__ y_in, T* lev,
                                                       int64_t lev_stride, int k, int n) {
  // staged columns: HX = 4 on each side of the tile (>= R, whole 16-byte vectors)
  constexpr int Hh = kTileY + 2 * R, HX = 4, WS = kTileX + 2 * HX;
  __shared__ __align__(16) T sh[3][Hh][WS];
  const TileLoc tl = tile_of(p);
  const ProbDev& q = p.probs[tl.prob];
  const SlotDev& s = p.slots[q.slot];
  if (k >= s.m) return;
  const int N = s.steps[k];
  if (n > N) return;
  const int nx = q.n[0], ny = q.n[1], nz = q.n[2];
  const int x0 = tl.tx * kTileX, y0 = tl.ty * kTileY, z = tl.z;
  const int64_t P = q.pts;
  const int64_t plane = (int64_t)z * nx * ny;
  const double hd = p.hk[tl.prob * GBS_MAX_SEQ + k];
  const T* yi = y_in + q.state_off;
  auto level = [&](int j) -> T* { return lev + (int64_t)j * lev_stride + q.state_off; };
  constexpr int F = 1 + DIM;
  const int x = x0 + threadIdx.x;
  if (n == 0) {
    if (x >= nx) return;
    const T h = T(hd);
    const T* f0 = static_cast<const T*>(p.f0) + q.state_off;
    T* d = level(1);
#pragma unroll
    for (int i = 0; i < kTileRows; ++i) {
      const int y = y0 + threadIdx.y + 8 * i;
      if (y >= ny) break;
      const int64_t pt = plane + (int64_t)y * nx + x;
#pragma unroll
      for (int fl = 0; fl < F; ++fl) d[fl * P + pt] = yi[fl * P + pt] + h * f0[fl * P + pt];
    }
    return;
  }
  const T* cur = level(n);
  const T* prev = (n == 1) ? yi : level(n - 1);
  T* dst = level(n + 1);
  // stage the level (vectors when kVec: every nx a multiple of 4, as in k_lf_tiled)
  if constexpr (kVec) {
    constexpr int VW = 16 / sizeof(T), GR = WS / VW, NV = Hh * GR, NITV = (NV + 255) / 256;
    using V = typename Vec16<T>::type;
    const int ltid = threadIdx.y * kTileX + threadIdx.x;
    V vs[3][NITV];
#pragma unroll
    for (int it = 0; it < NITV; ++it) {
      const int e = ltid + 256 * it;
      if (e < NV) {
        const int r = e / GR, g = e - r * GR;
        int gy = y0 - R + r;
        if (gy < 0 || gy >= ny) gy = wrap_any(gy, ny);
        int gx = x0 - HX + g * VW;
        if (gx < 0 || gx >= nx) gx = wrap_any(gx, nx);
        const T* a = cur + plane + (int64_t)gy * nx + gx;
#pragma unroll
        for (int f = 0; f < 3; ++f) vs[f][it] = __ldg(reinterpret_cast<const V*>(a + f * P));
      }
    }
#pragma unroll
    for (int it = 0; it < NITV; ++it) {
      const int e = ltid + 256 * it;
      if (e < NV) {
        const int r = e / GR, g = e - r * GR;
#pragma unroll
        for (int f = 0; f < 3; ++f) *reinterpret_cast<V*>(&sh[f][r][g * VW]) = vs[f][it];
      }
    }
  } else {
    using TS = TileStage<R>;
    T stg[3][TS::NIT];
#pragma unroll
    for (int it = 0; it < TS::NIT; ++it) {
      int r, cl;
      if (TS::rc(it, r, cl)) {
        const T* a = cur + TS::at(r, cl, x0, y0, nx, ny, plane);
        stg[0][it] = ldg(a);
        stg[1][it] = ldg(a + P);
        stg[2][it] = ldg(a + 2 * P);
      }
    }
#pragma unroll
    for (int it = 0; it < TS::NIT; ++it) {
      int r, cl;
      if (TS::rc(it, r, cl)) {
        sh[0][r][cl + HX - R] = stg[0][it];
        sh[1][r][cl + HX - R] = stg[1][it];
        sh[2][r][cl + HX - R] = stg[2][it];
      }
    }
  }
  __syncthreads();
  if (x >= nx) return;
  const T idx = T(q.inv_dx[0]), idy = T(q.inv_dx[1]), idz = T(q.inv_dx[2]);
  const T* kap = static_cast<const T*>(p.kappa) + q.media_off;
  const T* bmed = static_cast<const T*>(p.b) + q.media_off;
  const T h2 = T(2.0 * hd);
  // previous level and media of a row, loaded one row ahead of their use
  T nprev[F], nkv = T(0), nbv = T(0);
  auto fetch_row = [&](int i) {
    const int y = y0 + threadIdx.y + 8 * i;
    if (y >= ny) return;
    const int64_t pt = plane + (int64_t)y * nx + x;
#pragma unroll
    for (int fl = 0; fl < F; ++fl) nprev[fl] = prev[fl * P + pt];
    nkv = ldg(kap + pt);
    nbv = ldg(bmed + pt);
  };
  fetch_row(0);
#pragma unroll
  for (int i = 0; i < kTileRows; ++i) {
    const int ly = threadIdx.y + 8 * i;
    const int y = y0 + ly;
    if (y >= ny) break;
    T pv[F];
#pragma unroll
    for (int fl = 0; fl < F; ++fl) pv[fl] = nprev[fl];
    const T kv = nkv, bv = nbv;
    if (i + 1 < kTileRows) fetch_row(i + 1);
    const int r = ly + R, cc = threadIdx.x + HX;
    T sxu = T(0), sxp = T(0), syv = T(0), syp = T(0);
#pragma unroll
    for (int j = 1; j <= R; ++j) {
      const T a = T(fd_coef<R>(j));
      sxp += a * (sh[0][r][cc + j] - sh[0][r][cc - j]);
      sxu += a * (sh[1][r][cc + j] - sh[1][r][cc - j]);
      syp += a * (sh[0][r + j][cc] - sh[0][r - j][cc]);
      syv += a * (sh[2][r + j][cc] - sh[2][r - j][cc]);
    }
    const int64_t pt = plane + (int64_t)y * nx + x;
    T div = sxu * idx + syv * idy, szp = T(0);
    if (DIM == 3) {
      T szw = T(0);
#pragma unroll
      for (int j = 1; j <= R; ++j) {
        const int zp = z + j >= nz ? z + j - nz : z + j;
        const int zm = z - j < 0 ? z - j + nz : z - j;
        const int64_t op = (int64_t)(zp - z) * nx * ny, om = (int64_t)(zm - z) * nx * ny;
        const T a = T(fd_coef<R>(j));
        szp += a * (ldg(cur + pt + op) - ldg(cur + pt + om));
        szw += a * (ldg(cur + 3 * P + pt + op) - ldg(cur + 3 * P + pt + om));
      }
      div += szw * idz;
    }
    T f[kMaxFields];
    f[0] = -kv * div;
    f[1] = -bv * (sxp * idx);
    f[2] = -bv * (syp * idy);
    if (DIM == 3) f[3] = -bv * (szp * idz);
#pragma unroll
    for (int fl = 0; fl < F; ++fl) dst[fl * P + pt] = pv[fl] + h2 * f[fl];
  }
}

// Reverse step, tiled (same recursion as k_adj_rev):
//   M[j] = M[j+2] + init_j + 2h A^T M[j+1],  g += 2h mu_p (-div y_j),  mu = M[j+1],
// with A^T mu = (D.(b mu_vel), grad(kappa mu_p)).  The tile holds kappa mu_p, b mu_u, b mu_v
// of M[j+1] and, in FP32, y_j's u, v (the FP64 build takes div y_j through the cache to stay
// within 48 KB of static shared memory).
template <typename T, int DIM, int R>
__global__ void __launch_bounds__(256) k_adj_rev_tiled(const StepPlan p, const T* __restrict__ lev,
                                                       int64_t lev_stride, const T* __restrict__ lam_out, T* mA,
                                                       T* mB, double* grad, float2* gpair, int k, int jrev) {
  constexpr int W = kTileX + 2 * R, Hh = kTileY + 2 * R;
  constexpr bool kStageY = sizeof(T) == 4;
  constexpr int NS = kStageY ? 5 : 3;
  __shared__ T sh[NS][Hh][W + 1];
  const TileLoc tl = tile_of(p);
  const ProbDev& q = p.probs[tl.prob];
  const SlotDev& s = p.slots[q.slot];
  if (k >= s.m) return;
  const int N = s.steps[k];
  const int j = N + 1 - jrev;
  if (j < 1) return;
  const int nx = q.n[0], ny = q.n[1], nz = q.n[2];
  const int x0 = tl.tx * kTileX, y0 = tl.ty * kTileY, z = tl.z;
  const int64_t P = q.pts;
  const int64_t plane = (int64_t)z * nx * ny;
  constexpr int F = 1 + DIM;
  const double hd = p.hk[tl.prob * GBS_MAX_SEQ + k];
  const double c = s.c[k];
  T* dst = (((N + 1 - j) & 1) == 0 ? mA : mB) + q.state_off;
  const T* src = (((N + 1 - j) & 1) == 0 ? mB : mA) + q.state_off;   // M[j+1]
  const T* lo = lam_out + q.state_off;
  const int x = x0 + threadIdx.x;
  // per-thread constants (FP64 arithmetic is a small fraction of GB300's FP32 rate: none per point)
  const T wq = T(0.25 * c), wh = T(0.5 * c);               // seeds c/4 and c/2 of lam_out
  const T seed = j == N ? wh : j == N - 1 ? wq : T(0);
  const float h2hi = (float)(2.0 * hd), h2lo = (float)(2.0 * hd - (double)h2hi);
  if (j == N + 1) {
    if (x >= nx) return;
#pragma unroll
    for (int i = 0; i < kTileRows; ++i) {
      const int y = y0 + threadIdx.y + 8 * i;
      if (y >= ny) break;
      const int64_t pt = plane + (int64_t)y * nx + x;
#pragma unroll
      for (int fl = 0; fl < F; ++fl) dst[fl * P + pt] = wq * lo[fl * P + pt];
      if (kStageY && k == 0) gpair[q.media_off + pt] = make_float2(0.f, 0.f);   // start of the macro-step
    }
    return;
  }
  const T* kappa = static_cast<const T*>(p.kappa) + q.media_off;
  const T* bmed = static_cast<const T*>(p.b) + q.media_off;
  const T* yj = lev + (int64_t)j * lev_stride + q.state_off;
  using TS = TileStage<R>;
  T stg[NS + 2][TS::NIT];   // kappa, b, M[j+1] p, u, v, (y_j u, v)
#pragma unroll
  for (int it = 0; it < TS::NIT; ++it) {
    int r, cl;
    if (TS::rc(it, r, cl)) {
      const int64_t e = TS::at(r, cl, x0, y0, nx, ny, plane);
      stg[0][it] = ldg(kappa + e);
      stg[1][it] = ldg(bmed + e);
      stg[2][it] = ldg(src + e);
      stg[3][it] = ldg(src + P + e);
      stg[4][it] = ldg(src + 2 * P + e);
      if constexpr (kStageY) {
        stg[5][it] = ldg(yj + P + e);
        stg[6][it] = ldg(yj + 2 * P + e);
      }
    }
  }
#pragma unroll
  for (int it = 0; it < TS::NIT; ++it) {
    int r, cl;
    if (TS::rc(it, r, cl)) {
      sh[0][r][cl] = stg[0][it] * stg[2][it];
      sh[1][r][cl] = stg[1][it] * stg[3][it];
      sh[2][r][cl] = stg[1][it] * stg[4][it];
      if constexpr (kStageY) {
        sh[3][r][cl] = stg[5][it];
        sh[4][r][cl] = stg[6][it];
      }
    }
  }
  __syncthreads();
  if (x >= nx) return;
  const T idx = T(q.inv_dx[0]), idy = T(q.inv_dx[1]), idz = T(q.inv_dx[2]);
  const T h2 = T(2.0 * hd);
  // point-wise operands of a row, loaded one row ahead of their use: M[j+2] plus the seeds of
  // lam_out, and (FP32) mu_p and the gradient pair
  T nbase[F], nmu = T(0);
  float2 ngp = make_float2(0.f, 0.f);
  auto fetch_row = [&](int i) {
    const int y = y0 + threadIdx.y + 8 * i;
    if (y >= ny) return;
    const int64_t pt = plane + (int64_t)y * nx + x;
#pragma unroll
    for (int fl = 0; fl < F; ++fl) {
      const int64_t e = fl * P + pt;
      T base = (j <= N - 1) ? dst[e] : T(0);          // M[j+2]
      if (j >= N - 1) base += seed * lo[e];
      nbase[fl] = base;
    }
    if constexpr (kStageY) {
      nmu = ldg(src + pt);
      ngp = gpair[q.media_off + pt];
    }
  };
  fetch_row(0);
#pragma unroll
  for (int i = 0; i < kTileRows; ++i) {
    const int ly = threadIdx.y + 8 * i;
    const int y = y0 + ly;
    if (y >= ny) break;
    T base[F];
#pragma unroll
    for (int fl = 0; fl < F; ++fl) base[fl] = nbase[fl];
    const T mu_p = nmu;
    const float2 gp = ngp;
    if (i + 1 < kTileRows) fetch_row(i + 1);
    const int r = ly + R, cc = threadIdx.x + R;
    const int64_t pt = plane + (int64_t)y * nx + x;
    T sx_bu = T(0), sy_bv = T(0), sx_kp = T(0), sy_kp = T(0), sdx = T(0), sdy = T(0);
#pragma unroll
    for (int jj = 1; jj <= R; ++jj) {
      const T a = T(fd_coef<R>(jj));
      sx_kp += a * (sh[0][r][cc + jj] - sh[0][r][cc - jj]);
      sy_kp += a * (sh[0][r + jj][cc] - sh[0][r - jj][cc]);
      sx_bu += a * (sh[1][r][cc + jj] - sh[1][r][cc - jj]);
      sy_bv += a * (sh[2][r + jj][cc] - sh[2][r - jj][cc]);
      if constexpr (kStageY) {
        sdx += a * (sh[3][r][cc + jj] - sh[3][r][cc - jj]);
        sdy += a * (sh[4][r + jj][cc] - sh[4][r - jj][cc]);
      }
    }
    T at[kMaxFields];
    at[0] = sx_bu * idx + sy_bv * idy;
    at[1] = sx_kp * idx;
    at[2] = sy_kp * idy;
    T dv;
    if constexpr (kStageY) {
      dv = sdx * idx + sdy * idy;
    } else {
      const PointGeo g = geo_of(q, pt);
      T inv_dx[3] = {idx, idy, idz};
      dv = div_point<T, DIM, R>(yj, P, g, inv_dx);
    }
    if (DIM == 3) {
      T sz_bw = T(0), sz_kp = T(0), sdz = T(0);
#pragma unroll
      for (int jj = 1; jj <= R; ++jj) {
        const int zp = z + jj >= nz ? z + jj - nz : z + jj;
        const int zm = z - jj < 0 ? z - jj + nz : z - jj;
        const int64_t op = (int64_t)(zp - z) * nx * ny, om = (int64_t)(zm - z) * nx * ny;
        const T a = T(fd_coef<R>(jj));
        sz_bw += a * (ldg(bmed + pt + op) * ldg(src + 3 * P + pt + op) - ldg(bmed + pt + om) * ldg(src + 3 * P + pt + om));
        sz_kp += a * (ldg(kappa + pt + op) * ldg(src + pt + op) - ldg(kappa + pt + om) * ldg(src + pt + om));
        if constexpr (kStageY) sdz += a * (ldg(yj + 3 * P + pt + op) - ldg(yj + 3 * P + pt + om));
      }
      at[0] += sz_bw * idz;
      at[3] = sz_kp * idz;
      if constexpr (kStageY) dv += sdz * idz;
    }
#pragma unroll
    for (int fl = 0; fl < F; ++fl) dst[fl * P + pt] = base[fl] + h2 * at[fl];
    if constexpr (kStageY) {
      // FP32: gpair += 2h mu_p (-div y_j) in FP32 pairs (TwoProd by FMA, TwoSum); the finish
      // kernel folds the macro-step's sum into the FP64 gradient once.  GB300's FP64 pipe
      // would otherwise bound this kernel.
      const float mu = (float)mu_p, dvf = -(float)dv;
      const float pr = __fmul_rn(mu, dvf);
      const float pe = fmaf(mu, dvf, -pr);                        // mu * dvf = pr + pe exactly
      const float th = __fmul_rn(h2hi, pr);
      const float te = fmaf(h2hi, pe, fmaf(h2lo, pr, fmaf(h2hi, pr, -th)));
      const float2 acc = gp;
      const float sh = __fadd_rn(acc.x, th);
      const float bv = __fsub_rn(sh, acc.x);
      const float se = __fadd_rn(__fsub_rn(acc.x, __fsub_rn(sh, bv)), __fsub_rn(th, bv));
      const float lo2 = __fadd_rn(acc.y, __fadd_rn(se, te));
      const float hi2 = __fadd_rn(sh, lo2);
      gpair[q.media_off + pt] = make_float2(hi2, __fsub_rn(lo2, __fsub_rn(hi2, sh)));
    } else {
      grad[q.media_off + pt] += 2.0 * hd * (double)ldg(src + pt) * (-(double)dv);
    }
  }
}

// After the reverse sweep of sequence k: acc (+)= M[1] + M[2], shared (+)= h_k M[1].  The FP32
// build keeps acc as (hi, lo) float pairs in the same 8-byte slots (TwoSum accumulation), the
// FP64 build as doubles.
__device__ __forceinline__ float2 pair_add_f(float2 a, float b) {
  const float s = __fadd_rn(a.x, b);
  const float bb = __fsub_rn(s, a.x);
  const float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  const float lo = __fadd_rn(a.y, e);
  const float hi = __fadd_rn(s, lo);
  return make_float2(hi, __fsub_rn(lo, __fsub_rn(hi, s)));
}

template <typename T, int DIM>
__global__ void __launch_bounds__(kPlainBlock) k_adj_gather(const StepPlan p, const T* mA, const T* mB,
                                                            T* shared, int k) {
  const Loc L = locate(p);
  if (L.prob < 0) return;
  const ProbDev& q = p.probs[L.prob];
  const SlotDev& s = p.slots[q.slot];
  if (k >= s.m) return;
  constexpr int F = 1 + DIM;
  const double hd = p.hk[L.prob * GBS_MAX_SEQ + k];
  // M[1]: (N + 1 - 1) = N even -> buffer A; M[2] -> buffer B
  const T* m1 = mA + q.state_off;
  const T* m2 = mB + q.state_off;
  T* sh = shared + q.state_off;
  const bool first = (k == 0);
  const T hT = T(hd);
#pragma unroll
  for (int fl = 0; fl < F; ++fl) {
    const int64_t e = fl * q.pts + L.i;
    if constexpr (sizeof(T) == 4) {
      float2* acc = reinterpret_cast<float2*>(p.acc) + q.state_off;
      const float2 v = pair_add_f(make_float2(m1[e], 0.f), m2[e]);
      acc[e] = first ? v : pair_add_f(pair_add_f(acc[e], v.x), v.y);
    } else {
      double* acc = p.acc + q.state_off;
      const double v = (double)m1[e] + (double)m2[e];
      acc[e] = first ? v : acc[e] + v;
    }
    const T hv = hT * m1[e];
    sh[e] = first ? hv : sh[e] + hv;
  }
}

// lam_in = acc + A^T shared;  g += (shared)_p (-div y_in).
template <typename T, int DIM, int R>
__global__ void __launch_bounds__(kPlainBlock) k_adj_finish(const StepPlan p, const T* __restrict__ y_in,
                                                            const T* __restrict__ shared, T* lam_in,
                                                            double* grad, const float2* gpair) {
  const Loc L = locate(p);
  if (L.prob < 0) return;
  const ProbDev& q = p.probs[L.prob];
  constexpr int F = 1 + DIM;
  const PointGeo g = geo_of(q, L.i);
  T inv_dx[3];
  load_inv_dx(q, inv_dx);
  const T* kappa = static_cast<const T*>(p.kappa) + q.media_off;
  const T* bmed = static_cast<const T*>(p.b) + q.media_off;
  const T* sh = shared + q.state_off;
  T at[kMaxFields];
  rhs_T_point<T, DIM, R>(sh, q.pts, g, inv_dx, kappa, bmed, at);
  T* li = lam_in + q.state_off;
#pragma unroll
  for (int fl = 0; fl < F; ++fl) {
    const int64_t e = fl * q.pts + L.i;
    if constexpr (sizeof(T) == 4) {
      const float2 a = reinterpret_cast<const float2*>(p.acc)[q.state_off + e];
      li[e] = (a.x + at[fl]) + a.y;
    } else {
      li[e] = T(p.acc[q.state_off + e] + (double)at[fl]);
    }
  }
  const T dv = div_point<T, DIM, R>(y_in + q.state_off, q.pts, g, inv_dx);
  double gsum = (double)sh[L.i] * (-(double)dv);
  if (gpair) {   // the macro-step's reverse-step gradient terms (FP32 pairs, tiled kernels)
    const float2 gp = gpair[q.media_off + L.i];
    gsum += (double)gp.x + (double)gp.y;
  }
  grad[q.media_off + L.i] += gsum;
}

// Receiver injection; an index outside [0, n_pts) latches GBS_ERR_INVALID and is skipped.
template <typename T>
__global__ void k_inject(T* lam, const int64_t* idx, int n, const T* resid, int64_t n_pts, int* err) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int64_t i = idx[r];
  if (i < 0 || i >= n_pts) {
    atomicCAS(err, 0, (int)GBS_ERR_INVALID);
    return;
  }
  atomicAdd(lam + i, resid[r]);
}

// ---------------------------------------------------------------------------
// Host-side dispatch
// ---------------------------------------------------------------------------

// the tensor-map argument of launches that stage with loads (never read)
const CUtensorMap kNoTensorMap{};

template <typename T, int SYS, int DIM, int R>
int macro_step_t(const StepPlan& p, const SeqLevels& lv, const void* y_in_v, void* y_out_v, cudaStream_t st) {
  const T* y_in = static_cast<const T*>(y_in_v);
  auto* y_out = static_cast<typename out_of<T>::type*>(y_out_v);
  const dim3 grid((unsigned)p.total_blocks), block(kPlainBlock);
  int launches = 0;
  k_f0<T, SYS, DIM, R><<<grid, block, 0, st>>>(p, y_in);
  ++launches;
  if constexpr (std::is_same<T, float>::value && SYS == SYS_ACOUSTIC && DIM >= 2) {
    if (lv.base) {
      // sequence-fused: every scheduled sequence has its own level pair; the Forward-Euler
      // levels, then one launch per leap-frog level n advancing every sequence that has it
      int nmax = 0;
      for (int k = 0; k < p.max_m; ++k) {
        if (!((p.seq_mask >> k) & 1u)) continue;
        StepPlan q = p;
        q.L1 = static_cast<float*>(lv.base) + (2 * k + 1) * lv.stride;
        k_fe<T, SYS, DIM><<<grid, block, 0, st>>>(q, y_in, k);
        ++launches;
        nmax = std::max(nmax, p.max_steps_k[k]);
      }
      for (int n = 1; n <= nmax; ++n) {
        uint32_t all = 0;
        for (int k = 0; k < p.max_m; ++k)
          if (((p.seq_mask >> k) & 1u) && p.max_steps_k[k] >= n) all |= 1u << k;
        while (all) {
          // the next group of at most lv.group sequences
          uint32_t kmask = 0;
          for (int c = 0; all && (lv.group <= 0 || c < lv.group); ++c) {
            kmask |= all & (0u - all);
            all &= all - 1;
          }
          double bytes = 0.0;
          int64_t any = 0;
          for (int k = 0; k < p.max_m; ++k) {
            if (!((kmask >> k) & 1u)) continue;
            const int64_t pts = p.active_pts[k * (GBS_MAX_STEPS + 1) + n];
            // per sequence: y_(n-1) and y_n read, y_(n+1) written; f0 and the media once per
            // point for the group (the problems of its largest sequence count, exact for a
            // single problem or one weight slot)
            bytes += 12.0 * p.F * (double)pts;
            any = std::max(any, pts);
          }
          bytes += 4.0 * (p.F + 2) * (double)any;
          const int na = __builtin_popcount(kmask);
          const int u = timing_begin(p, st);
          if (p.nx_vec && lv.tmap)
            k_lf_tiled_seqs<T, DIM, R, true, true><<<(unsigned)(p.total_tiles * na), dim3(kTileX, 8), 0, st>>>(
                p, y_in, y_out, kmask, na, n, *static_cast<const CUtensorMap*>(lv.tmap), lv);
          else if (p.nx_vec)
            k_lf_tiled_seqs<T, DIM, R, true, false><<<(unsigned)(p.total_tiles * na), dim3(kTileX, 8), 0, st>>>(
                p, y_in, y_out, kmask, na, n, kNoTensorMap, lv);
          else
            k_lf_tiled_seqs<T, DIM, R, false, false><<<(unsigned)(p.total_tiles * na), dim3(kTileX, 8), 0, st>>>(
                p, y_in, y_out, kmask, na, n, kNoTensorMap, lv);
          timing_end(p, u, st, p.tev ? bytes : 0.0);
          ++launches;
        }
      }
      if (cudaPeekAtLastError() != cudaSuccess) return -1;
      return launches;
    }
  }
  for (int k = 0; k < p.max_m; ++k) {
    if (!((p.seq_mask >> k) & 1u)) continue;   // a partial step leaves this sequence to another rank
    k_fe<T, SYS, DIM><<<grid, block, 0, st>>>(p, y_in, k);
    ++launches;
    for (int n = 1; n <= p.max_steps_k[k]; ++n) {
      const int u = timing_begin(p, st);
      if constexpr (SYS == SYS_ACOUSTIC && DIM >= 2 && std::is_same<T, dsf>::value)
        p.nx_vec ? k_lf_tiled_x2<(DIM >= 2 ? DIM : 2), R, true><<<(unsigned)p.total_tiles, dim3(kTileX, 8), 0, st>>>(p, y_in, y_out, k, n)
                 : k_lf_tiled_x2<(DIM >= 2 ? DIM : 2), R, false><<<(unsigned)p.total_tiles, dim3(kTileX, 8), 0, st>>>(p, y_in, y_out, k, n);
      else if (SYS == SYS_ACOUSTIC && DIM >= 2 && p.nx_vec) {
        // the level staged by step n is L1 for odd n, else L0 (see k_lf_tiled)
        const void* map = p.lf_tmap[n & 1];
        bool tma = false;
        if constexpr (std::is_same<T, float>::value) {
          if (map) {
            k_lf_tiled<T, (DIM >= 2 ? DIM : 2), R, true, true><<<(unsigned)p.total_tiles, dim3(kTileX, 8), 0, st>>>(
                p, y_in, y_out, k, n, *static_cast<const CUtensorMap*>(map));
            tma = true;
          }
        }
        if (!tma)
          k_lf_tiled<T, (DIM >= 2 ? DIM : 2), R, true, false><<<(unsigned)p.total_tiles, dim3(kTileX, 8), 0, st>>>(
              p, y_in, y_out, k, n, kNoTensorMap);
      } else if (SYS == SYS_ACOUSTIC && DIM >= 2)
        k_lf_tiled<T, (DIM >= 2 ? DIM : 2), R, false, false><<<(unsigned)p.total_tiles, dim3(kTileX, 8), 0, st>>>(
            p, y_in, y_out, k, n, kNoTensorMap);
      else
        k_lf<T, SYS, DIM, R><<<grid, block, 0, st>>>(p, y_in, y_out, k, n);
      timing_end(p, u, st, p.tev ? p.unit_bytes * (double)p.active_pts[k * (GBS_MAX_STEPS + 1) + n] : 0.0);
      ++launches;
    }
  }
  if (cudaPeekAtLastError() != cudaSuccess) return -1;
  return launches;
}

template <typename T, int DIM, int R>
int adjoint_step_t(const AdjPlan& a, const void* y_in_v, const void* lam_out_v, void* lam_in_v,
                   double* grad, const int64_t* rcv_idx, int n_rcv, const void* rcv_resid,
                   cudaStream_t st) {
  const StepPlan& p = a.fw;
  const T* y_in = static_cast<const T*>(y_in_v);
  const T* lam_out = static_cast<const T*>(lam_out_v);
  T* lam_in = static_cast<T*>(lam_in_v);
  T* lev = static_cast<T*>(a.levels);
  const int64_t lev_stride = p.state_elems;
  T* mA = static_cast<T*>(a.mu0);
  T* mB = static_cast<T*>(a.mu1);
  T* shared = static_cast<T*>(a.shared);
  const dim3 grid((unsigned)p.total_blocks), block(kPlainBlock);
  const dim3 tgrid((unsigned)p.total_tiles), tblock(kTileX, 8);
  int launches = 0;
  k_f0<T, SYS_ACOUSTIC, DIM, R><<<grid, block, 0, st>>>(p, y_in);
  ++launches;
  for (int k = 0; k < p.max_m; ++k) {
    const int Nk = p.max_steps_k[k];
    for (int n = 0; n <= Nk; ++n) {
      if (DIM >= 2)
        p.nx_vec ? k_adj_fwd_tiled<T, DIM, R, true><<<tgrid, tblock, 0, st>>>(p, y_in, lev, lev_stride, k, n)
                 : k_adj_fwd_tiled<T, DIM, R, false><<<tgrid, tblock, 0, st>>>(p, y_in, lev, lev_stride, k, n);
      else
        k_adj_fwd<T, DIM, R><<<grid, block, 0, st>>>(p, y_in, lev, lev_stride, k, n);
      ++launches;
    }
    for (int t = 0; t <= Nk; ++t) {
      const int u = t > 0 ? timing_begin(p, st) : -1;
      if (DIM >= 2)
        k_adj_rev_tiled<T, DIM, R><<<tgrid, tblock, 0, st>>>(p, lev, lev_stride, lam_out, mA, mB, grad, a.gpair, k, t);
      else
        k_adj_rev<T, DIM, R><<<grid, block, 0, st>>>(p, y_in, lev, lev_stride, lam_out, mA, mB, grad, k, t);
      if (t > 0)
        timing_end(p, u, st, p.tev ? p.adj_unit_bytes * (double)p.active_pts[k * (GBS_MAX_STEPS + 1) + t] : 0.0);
      ++launches;
    }
    k_adj_gather<T, DIM><<<grid, block, 0, st>>>(p, mA, mB, shared, k);
    ++launches;
  }
  k_adj_finish<T, DIM, R><<<grid, block, 0, st>>>(p, y_in, shared, lam_in, grad,
                                                  (DIM >= 2 && sizeof(T) == 4) ? a.gpair : nullptr);
  ++launches;
  if constexpr (!std::is_same<T, dsf>::value) {   // pairs: the caller injects into the FP64 lam_in
    if (n_rcv > 0) {
      k_inject<T><<<(n_rcv + 127) / 128, 128, 0, st>>>(lam_in, rcv_idx, n_rcv, static_cast<const T*>(rcv_resid),
                                                       a.rcv_pts, a.err);
      ++launches;
    }
  }
  if (cudaPeekAtLastError() != cudaSuccess) return -1;
  return launches;
}

template <typename T>
int macro_step_sys(const StepPlan& p, const SeqLevels& lv, const void* yi, void* yo, cudaStream_t s) {
  if (p.system == GBS_WAVE1D) {
    return p.R == 2 ? macro_step_t<T, SYS_WAVE1D, 1, 2>(p, lv, yi, yo, s)
                    : macro_step_t<T, SYS_WAVE1D, 1, 3>(p, lv, yi, yo, s);
  }
  switch (p.ndim * 10 + p.R) {
    case 12: return macro_step_t<T, SYS_ACOUSTIC, 1, 2>(p, lv, yi, yo, s);
    case 13: return macro_step_t<T, SYS_ACOUSTIC, 1, 3>(p, lv, yi, yo, s);
    case 22: return macro_step_t<T, SYS_ACOUSTIC, 2, 2>(p, lv, yi, yo, s);
    case 23: return macro_step_t<T, SYS_ACOUSTIC, 2, 3>(p, lv, yi, yo, s);
    case 32: return macro_step_t<T, SYS_ACOUSTIC, 3, 2>(p, lv, yi, yo, s);
    case 33: return macro_step_t<T, SYS_ACOUSTIC, 3, 3>(p, lv, yi, yo, s);
  }
  return -1;
}

template <typename T>
int adjoint_sys(const AdjPlan& a, const void* yi, const void* lo, void* li, double* g,
                const int64_t* ri, int nr, const void* rr, cudaStream_t s) {
  switch (a.fw.ndim * 10 + a.fw.R) {
    case 12: return adjoint_step_t<T, 1, 2>(a, yi, lo, li, g, ri, nr, rr, s);
    case 13: return adjoint_step_t<T, 1, 3>(a, yi, lo, li, g, ri, nr, rr, s);
    case 22: return adjoint_step_t<T, 2, 2>(a, yi, lo, li, g, ri, nr, rr, s);
    case 23: return adjoint_step_t<T, 2, 3>(a, yi, lo, li, g, ri, nr, rr, s);
    case 32: return adjoint_step_t<T, 3, 2>(a, yi, lo, li, g, ri, nr, rr, s);
    case 33: return adjoint_step_t<T, 3, 3>(a, yi, lo, li, g, ri, nr, rr, s);
  }
  return -1;
}

}  // namespace

namespace {
template <typename T>
int f0_sys(const StepPlan& p, const void* yi, cudaStream_t st) {
  const dim3 grid((unsigned)p.total_blocks), block(kPlainBlock);
  const T* y = static_cast<const T*>(yi);
  if (p.system == GBS_WAVE1D) {
    if (p.R == 2) k_f0<T, SYS_WAVE1D, 1, 2><<<grid, block, 0, st>>>(p, y);
    else k_f0<T, SYS_WAVE1D, 1, 3><<<grid, block, 0, st>>>(p, y);
  } else {
    switch (p.ndim * 10 + p.R) {
      case 12: k_f0<T, SYS_ACOUSTIC, 1, 2><<<grid, block, 0, st>>>(p, y); break;
      case 13: k_f0<T, SYS_ACOUSTIC, 1, 3><<<grid, block, 0, st>>>(p, y); break;
      case 22: k_f0<T, SYS_ACOUSTIC, 2, 2><<<grid, block, 0, st>>>(p, y); break;
      case 23: k_f0<T, SYS_ACOUSTIC, 2, 3><<<grid, block, 0, st>>>(p, y); break;
      case 32: k_f0<T, SYS_ACOUSTIC, 3, 2><<<grid, block, 0, st>>>(p, y); break;
      case 33: k_f0<T, SYS_ACOUSTIC, 3, 3><<<grid, block, 0, st>>>(p, y); break;
      default: return -1;
    }
  }
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}
}  // namespace

int launch_f0(const StepPlan& p, const void* y_in, cudaStream_t s) {
  return p.f64 ? f0_sys<double>(p, y_in, s) : f0_sys<float>(p, y_in, s);
}

// FP64 -> FP32 pairs (nearest pair) for the GBS_F32X2 path
__global__ void k_to_ds(const double* __restrict__ a, dsf* __restrict__ o, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    o[i] = dsf(a[i]);
}

int ds_prologue(const StepPlan& p, const void* y_in, void* y_pairs, void* f0_pairs, cudaStream_t s) {
  k_to_ds<<<1024, 256, 0, s>>>(static_cast<const double*>(y_in), static_cast<dsf*>(y_pairs), p.state_elems);
  const int64_t m = p.probs_media_elems;
  k_to_ds<<<1024, 256, 0, s>>>(static_cast<const double*>(p.kappa), static_cast<dsf*>(p.ds_kappa), m);
  k_to_ds<<<1024, 256, 0, s>>>(static_cast<const double*>(p.b), static_cast<dsf*>(p.ds_b), m);
  StepPlan q = p;
  q.kappa = p.ds_kappa;
  q.b = p.ds_b;
  q.f0 = f0_pairs;
  q.f0_aux = nullptr;
  return f0_sys<dsf>(q, y_pairs, s) < 0 ? -1 : 4;
}

int plain_macro_step(const StepPlan& p, const void* y_in, void* y_out, cudaStream_t s) {
  if (p.system == GBS_ONEWAY_SPECTRAL) return spectral_macro_step(p, y_in, y_out, s);
  if (p.ds) {
    // the step reads y_in, kappa and b as FP32 pairs converted here, and writes FP64 y_out
    k_to_ds<<<1024, 256, 0, s>>>(static_cast<const double*>(y_in), static_cast<dsf*>(p.ds_y0), p.state_elems);
    int extra = 1;
    StepPlan q = p;
    if (p.system == GBS_ACOUSTIC) {
      const int64_t m = p.probs_media_elems;
      k_to_ds<<<1024, 256, 0, s>>>(static_cast<const double*>(p.kappa), static_cast<dsf*>(p.ds_kappa), m);
      k_to_ds<<<1024, 256, 0, s>>>(static_cast<const double*>(p.b), static_cast<dsf*>(p.ds_b), m);
      q.kappa = p.ds_kappa;
      q.b = p.ds_b;
      extra += 2;
    }
    const int l = macro_step_sys<dsf>(q, SeqLevels{nullptr, 0, nullptr}, p.ds_y0, y_out, s);
    return l < 0 ? l : l + extra;
  }
  const SeqLevels none{nullptr, 0, nullptr};
  return p.f64 ? macro_step_sys<double>(p, none, y_in, y_out, s) : macro_step_sys<float>(p, none, y_in, y_out, s);
}

int plain_macro_step_seqfused(const StepPlan& p, const SeqLevels& lv, const void* y_in, void* y_out, cudaStream_t s) {
  if (p.system != GBS_ACOUSTIC || p.ndim < 2 || p.f64 || p.ds || !lv.base) return plain_macro_step(p, y_in, y_out, s);
  return macro_step_sys<float>(p, lv, y_in, y_out, s);
}

int inject(int f64, void* lam, const int64_t* idx, int n, const void* values, int64_t n_valid, int* err,
           cudaStream_t s) {
  if (n <= 0) return 0;
  if (f64)
    k_inject<double><<<(n + 127) / 128, 128, 0, s>>>(static_cast<double*>(lam), idx, n,
                                                      static_cast<const double*>(values), n_valid, err);
  else
    k_inject<float><<<(n + 127) / 128, 128, 0, s>>>(static_cast<float*>(lam), idx, n,
                                                     static_cast<const float*>(values), n_valid, err);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

namespace {
// FP32 pairs -> FP64 (exact: a pair's value is the FP64 sum of its parts)
__global__ void k_from_ds(const dsf* __restrict__ a, double* __restrict__ o, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    o[i] = double(a[i]);
}
}  // namespace

int plain_adjoint_step_pairs(const AdjPlan& a, void* lam_pairs, const void* y_in, const void* lam_out, void* lam_in,
                             double* grad_kappa, const int64_t* rcv_idx, int n_rcv, const void* rcv_resid,
                             cudaStream_t s) {
  const StepPlan& p = a.fw;
  if (p.system != GBS_ACOUSTIC || !p.ds || !lam_pairs) return -1;
  // y_in, kappa, b and lam_out as FP32 pairs; the adjoint macro-step in pair arithmetic with
  // lam_in written over the pair copy of lam_out (read only by the reverse steps before it)
  const int64_t E = p.state_elems, M = p.probs_media_elems;
  k_to_ds<<<1024, 256, 0, s>>>(static_cast<const double*>(y_in), static_cast<dsf*>(p.ds_y0), E);
  k_to_ds<<<1024, 256, 0, s>>>(static_cast<const double*>(p.kappa), static_cast<dsf*>(p.ds_kappa), M);
  k_to_ds<<<1024, 256, 0, s>>>(static_cast<const double*>(p.b), static_cast<dsf*>(p.ds_b), M);
  k_to_ds<<<1024, 256, 0, s>>>(static_cast<const double*>(lam_out), static_cast<dsf*>(lam_pairs), E);
  AdjPlan b = a;
  b.fw.kappa = p.ds_kappa;
  b.fw.b = p.ds_b;
  const int l = adjoint_sys<dsf>(b, p.ds_y0, lam_pairs, lam_pairs, grad_kappa, nullptr, 0, nullptr, s);
  if (l < 0) return -1;
  k_from_ds<<<1024, 256, 0, s>>>(static_cast<const dsf*>(lam_pairs), static_cast<double*>(lam_in), E);
  int extra = 5;
  if (n_rcv > 0) {
    if (inject(1, lam_in, rcv_idx, n_rcv, rcv_resid, a.rcv_pts, a.err, s) < 0) return -1;
    ++extra;
  }
  if (cudaPeekAtLastError() != cudaSuccess) return -1;
  return l + extra;
}

int plain_adjoint_step(const AdjPlan& a, const void* y_in, const void* lam_out, void* lam_in,
                       double* grad_kappa, const int64_t* rcv_idx, int n_rcv,
                       const void* rcv_resid, cudaStream_t s) {
  if (a.fw.system != GBS_ACOUSTIC) return -1;
  return a.fw.f64 ? adjoint_sys<double>(a, y_in, lam_out, lam_in, grad_kappa, rcv_idx, n_rcv, rcv_resid, s)
                  : adjoint_sys<float>(a, y_in, lam_out, lam_in, grad_kappa, rcv_idx, n_rcv, rcv_resid, s);
}


int lf_tma_encode(void* map, void* base, int nx, int ny, int nz, int F, int R) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    looked_up = true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    else
      cudaGetLastError();
  }
  if (!encode || nx % 4 || F < 3 || (reinterpret_cast<uintptr_t>(base) & 15)) return -1;
  // dimensions x, y, z, field; strides of y, z and field in bytes (multiples of 16: nx % 4 == 0)
  const cuuint64_t dims[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)F};
  const cuuint64_t strides[3] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4, (cuuint64_t)nx * ny * nz * 4};
  // the staging box of k_lf_tiled: HX = 4 columns on either side of the 32-column tile, R rows
  // above and below its 32 rows, one z-plane, the fields p, u, v
  const cuuint32_t box[4] = {(cuuint32_t)(kTileX + 8), (cuuint32_t)(kTileY + 2 * R), 1, 3};
  const cuuint32_t elem[4] = {1, 1, 1, 1};
  const CUresult r = encode(static_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides,
                            box, elem, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : -1;
}

}  // namespace gbs

namespace gbs {
namespace {
template <typename T>
__global__ void __launch_bounds__(256) k_finish_partial(const T* y_in, const double* __restrict__ total, T* y_out,
                                                        int64_t n, int inc) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    y_out[e] = T(inc ? (double)y_in[e] + total[e] : total[e]);
}
}  // namespace

// The end of a sequence-parallel macro-step: total is the FP64 sum of every rank's combine share;
// FP32 states (increment form) add y_in, FP64 and FP32-pair states hold sum_k c_k y*_k already.
int finish_partial(const StepPlan& p, const void* y_in, const double* total, void* y_out, cudaStream_t s) {
  if (p.f64)
    k_finish_partial<double><<<1024, 256, 0, s>>>(static_cast<const double*>(y_in), total, static_cast<double*>(y_out),
                                                  p.state_elems, 0);
  else
    k_finish_partial<float><<<1024, 256, 0, s>>>(static_cast<const float*>(y_in), total, static_cast<float*>(y_out),
                                                 p.state_elems, 1);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}
}  // namespace gbs
