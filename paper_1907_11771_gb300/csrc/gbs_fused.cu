// Time-blocked FP32 macro-step for 2D acoustics: a persistent dataflow kernel.
//
// One macro-step (Sec. 2.1 eq. "GBS", Sec. 3.6, Sec. 3.2) runs as
//   1. f0 = f(y_in)              point-parallel, shared by every sequence (Sec. 3.6)
//   2. k_passes                  all Forward-Euler / leap-frog levels of all sequences
//   3. k_combine                 y_out = sum_k c_k y*_k, an FP64 sum of the averages
//
// Work items.  Sequence k has the Forward-Euler level y_1 and N_k leap-frog
// levels y_2 .. y_(N+1).  The leap-frog levels are cut into passes of
// T in {2, 4, 6, 8} levels (the first pass takes N mod 8, the others 8), and
// every pass into tiles: strips of at most 128 columns times segments of rows.
// An item (problem, k, pass, tile) reads the two levels (y_(n-1), y_n) of the
// previous pass over its tile plus an R*T halo, advances them T levels and
// writes (y_(n+T-1), y_(n+T)) -- or, in the sequence's last pass, the average
// y*_k = (y_(N-1) + 2 y_N + y_(N+1)) / 4 -- for its tile.  The first pass
// starts from (y_0, y_1 = y_0 + h f0).  Passes alternate between two buffer
// sets, so an item never overwrites data a neighbour may still read, and an
// item waits (bounded spin, then GBS_ERR_TIMEOUT) until the previous pass is
// done on the 3 x 3 neighbouring tiles.  Items are dequeued from one atomic
// counter in an order where every dependency comes first, so the kernel makes
// progress with any grid size.
//
// Inside an item (one CTA, one grid column per thread) the tile is swept row
// by row with a time skew: at sweep step s, level t computes local row
// s - R T - R t.  Every level keeps the last 2R+1 rows of p and v of its
// thread's column in registers (the y-stencils and the leap-frog "previous"
// value) and publishes its newest row of p and u in a shared-memory ring of
// 2R+1 rows, from which the neighbouring columns take their x-stencils.  One
// __syncthreads per sweep step orders the ring traffic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "gbs_internal.h"
#include "gbs_stencil.cuh"

namespace gbs {
namespace fused {

#ifndef GBS_FUSED_TMAX
#define GBS_FUSED_TMAX 4           // longest pass; 4 keeps 2 CTAs per SM
#endif
constexpr int kThreads = 256;      // strip width including the halo: one column per thread
constexpr int kTMax = GBS_FUSED_TMAX;  // leap-frog levels per pass (even)
constexpr int kMinBlocks = kTMax <= 4 ? 2 : 1;
constexpr int kMaxDeps = 9;
constexpr int kMaxPasses = GBS_MAX_STEPS / 2 + 2;
constexpr long long kSpinLimit = 1ll << 20;   // default: about half a second of polling

struct Item {
  int prob, seq, pass, tile;
};

// Per (slot, sequence, pass).
struct PassDesc {
  int T;      // leap-frog levels in this pass
  int first;  // level 0 is y_1 = y_0 + h f0 and level -1 is y_0
  int last;   // writes the average y* instead of two levels
  int pad;
};

// Strips and row segments of one problem.  Strip sx covers columns
// [sx nx / nst, (sx+1) nx / nst) and segment sy rows [sy ny / nseg, (sy+1) ny / nseg),
// so sizes differ by at most one; every strip and segment is at least as wide
// as the R*T halo unless it is the only one.
struct TileGeo {
  int nst, nseg;
  int pad0, pad1;
};

struct Params {
  const Item* items;
  const int* deps;
  int n_items;
  int* done;
  int* queue;
  int* err;
  const ProbDev* probs;
  const SlotDev* slots;
  const double* hk;
  const float2* hkf;
  const float* kappa;
  const float* b;
  const float* y0;
  const float* f0;
  float* lev;            // [seq][set][2][E]
  float* ystar;          // [seq][E]
  int64_t E;
  const PassDesc* pdesc; // [slot][seq][pass]
  const TileGeo* tgeo;   // per problem
  long long spin_limit;  // polls of a dependency flag before GBS_ERR_TIMEOUT
};

__device__ __forceinline__ int wrapi(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

// a mod n for -2n <= a < 3n (rows and columns never stray further from the tile)
__device__ __forceinline__ int wrapf(int a, int n) {
  if (a >= n) a -= n;
  if (a >= n) a -= n;
  if (a < 0) a += n;
  if (a < 0) a += n;
  return a;
}

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// x-derivative sum over a ring row (shared memory), unscaled
template <int R>
__device__ __forceinline__ float dsum(const float* row, int xs) {
  float s = 0.f;
#pragma unroll
  for (int j = 1; j <= R; ++j) s += float(fd_coef<R>(j)) * (row[xs + j] - row[xs - j]);
  return s;
}

// y-derivative sum over a register window indexed by row mod (2R+1), unscaled
template <int R>
__device__ __forceinline__ float dwin(const float (&w)[2 * R + 1], int c) {
  constexpr int U = 2 * R + 1;
  float s = 0.f;
#pragma unroll
  for (int j = 1; j <= R; ++j) s += float(fd_coef<R>(j)) * (w[(c + j) % U] - w[(c + U - j) % U]);
  return s;
}

// Shared memory of one CTA: level rings of (p, u) pairs [T_MAX][UR][kRow] followed by media
// rings of (kappa, b) pairs [M][kRow].  Rows are padded by kPad on both sides so the
// x-stencil of every thread (including the halo columns, whose values are discarded) stays
// inside the row.  The CTA synchronises once every kSyncEvery sweep steps, so a ring must
// hold 2R + kSyncEvery rows of a level (readers lag up to 2R rows behind the writer) and the
// media ring R T_MAX + kSyncEvery + 1 rows.
constexpr int kPad = 4;
constexpr int kRow = kThreads + 2 * kPad;
constexpr int kSyncEvery = 2;

template <int R>
__host__ __device__ constexpr int ring_rows() { return 2 * R + kSyncEvery; }
template <int R>
__host__ __device__ constexpr int media_rows() { return R * kTMax + kSyncEvery + 1; }

// x-derivative sums of p and u at once from a ring row of (p, u) pairs, unscaled
template <int R>
__device__ __forceinline__ float2 dsum2(const float2* row) {
  float sp = 0.f, su = 0.f;
#pragma unroll
  for (int j = 1; j <= R; ++j) {
    const float2 a = row[j], b = row[-j];
    sp += float(fd_coef<R>(j)) * (a.x - b.x);
    su += float(fd_coef<R>(j)) * (a.y - b.y);
  }
  return make_float2(sp, su);
}

template <int R, int T>
__device__ __forceinline__ void run_item(const Params& P, const Item& it, const PassDesc& pd, float* smem) {
  constexpr int U = 2 * R + 1;       // register window rows
  constexpr int UR = ring_rows<R>();  // shared ring rows per level
  constexpr int M = media_rows<R>();
  constexpr int OFF = 64 * U;        // keeps compile-time slot arithmetic non-negative
  const int tid = threadIdx.x;
  const ProbDev q = P.probs[it.prob];
  const TileGeo tg = P.tgeo[it.prob];
  const int nx = q.n[0], ny = q.n[1];
  const int sx = it.tile % tg.nst, sy = it.tile / tg.nst;
  const int x0 = (sx * nx) / tg.nst;
  const int wout = ((sx + 1) * nx) / tg.nst - x0;
  const int Y0 = (sy * ny) / tg.nseg;
  const int hs = ((sy + 1) * ny) / tg.nseg - Y0;
  const int x = wrapi(x0 - R * T + tid, nx);
  const float2 hf = P.hkf[it.prob * GBS_MAX_SEQ + it.seq];
  const float h1 = hf.x, h2 = hf.y;
  const float h2x = h2 * float(q.inv_dx[0]), h2y = h2 * float(q.inv_dx[1]);
  const float rxy = float(q.inv_dx[1] / q.inv_dx[0]);   // y-stencil weight relative to x
  const int64_t PP = q.pts;
  const float* kap = P.kappa + q.media_off;
  const float* bb = P.b + q.media_off;
  const float* inA;
  const float* inB;
  if (pd.first) {
    inA = P.y0 + q.state_off;   // level -1 = y_0
    inB = P.f0 + q.state_off;   // level 0 = y_0 + h f0
  } else {
    const int set_in = (it.pass - 1) & 1;
    inA = P.lev + ((int64_t)(it.seq * 2 + set_in) * 2 + 0) * P.E + q.state_off;
    inB = P.lev + ((int64_t)(it.seq * 2 + set_in) * 2 + 1) * P.E + q.state_off;
  }
  float* outA;
  float* outB = nullptr;
  if (pd.last) {
    outA = P.ystar + (int64_t)it.seq * P.E + q.state_off;
  } else {
    const int set_out = it.pass & 1;
    outA = P.lev + ((int64_t)(it.seq * 2 + set_out) * 2 + 0) * P.E + q.state_off;
    outB = P.lev + ((int64_t)(it.seq * 2 + set_out) * 2 + 1) * P.E + q.state_off;
  }
  const bool out_col = tid >= R * T && tid < R * T + wout;
  float2* const lvl = reinterpret_cast<float2*>(smem) + kPad + tid;               // this column
  float2* const med = reinterpret_cast<float2*>(smem) + kTMax * UR * kRow + kPad + tid;
  auto RING = [&](int t, int slot) -> float2* { return lvl + (t * UR + slot) * kRow; };

  float wp[T][U], wv[T][U];
#pragma unroll
  for (int t = 0; t < T; ++t)
#pragma unroll
    for (int u = 0; u < U; ++u) wp[t][u] = wv[t][u] = 0.f;

  // global loads of one sweep step, issued one step ahead
  const int S = hs + 2 * R * T;
  int gy0 = wrapf(Y0 - R * T, ny);          // grid row of level 0 at step 0
  int gy1 = wrapf(Y0 - R * T - R, ny);      // grid row of level -1 (level 1's row) at step 0
  float n0p, n0u, n0v, n1p = 0.f, n1u = 0.f, n1v = 0.f, nk, nb;
  auto fetch = [&](int s) {
    const int64_t e0 = (int64_t)gy0 * nx + x;
    if (pd.first) {
      n0p = __ldg(inA + e0) + h1 * __ldg(inB + e0);
      n0u = __ldg(inA + PP + e0) + h1 * __ldg(inB + PP + e0);
      n0v = __ldg(inA + 2 * PP + e0) + h1 * __ldg(inB + 2 * PP + e0);
    } else {
      n0p = __ldcg(inB + e0);
      n0u = __ldcg(inB + PP + e0);
      n0v = __ldcg(inB + 2 * PP + e0);
    }
    nk = __ldg(kap + e0);
    nb = __ldg(bb + e0);
    if (s >= 2 * R) {
      const int64_t e1 = (int64_t)gy1 * nx + x;
      if (pd.first) {
        n1p = __ldg(inA + e1);
        n1u = __ldg(inA + PP + e1);
        n1v = __ldg(inA + 2 * PP + e1);
      } else {
        n1p = __ldcg(inA + e1);
        n1u = __ldcg(inA + PP + e1);
        n1v = __ldcg(inA + 2 * PP + e1);
      }
    }
  };
  fetch(0);
  int ms0 = 0;   // media ring slot of level 0's row
  int rs0 = 0;   // level ring slot of level 0's row
  for (int sb = 0; sb < S; sb += U) {
#pragma unroll
    for (int uu = 0; uu < U; ++uu) {
      const int s = sb + uu;
      if (s >= S) break;
      // ---- commit level 0 (local row s - R T), level -1, media ----
      const int slot0 = (uu + OFF - R * T) % U;
      const float p0 = n0p, u0 = n0u, v0 = n0v;
      const float am_p = n1p, am_u = n1u, am_v = n1v;
      wp[0][slot0] = p0;
      wv[0][slot0] = v0;
      RING(0, rs0)[0] = make_float2(p0, u0);
      med[ms0 * kRow] = make_float2(nk, nb);
      // ---- prefetch step s + 1 ----
      gy0 = gy0 + 1 == ny ? 0 : gy0 + 1;
      gy1 = gy1 + 1 == ny ? 0 : gy1 + 1;
      if (s + 1 < S) fetch(s + 1);
      // ---- levels 1..T: level t computes local row s - R T - R t ----
#pragma unroll
      for (int t = 1; t <= T; ++t) {
        if (s >= 2 * t * R) {
          const int sl = (uu + OFF - R * T - R * t) % U;   // register window slot of this row
          int rs = rs0 - R * t;                             // ring slot of this row
          if (rs < 0) rs += UR;
          if (rs < 0) rs += UR;
          int ms = ms0 - R * t;
          if (ms < 0) ms += M;
          const float2 kb = med[ms * kRow];
          const float2 sxpu = dsum2<R>(RING(t - 1, rs));
          const float syp = dwin<R>(wp[t - 1], sl);
          const float syv = dwin<R>(wv[t - 1], sl);
          float pp, pu, pv;
          if (t == 1) {
            pp = am_p;
            pu = am_u;
            pv = am_v;
          } else {
            pp = wp[t - 2][sl];
            pv = wv[t - 2][sl];
            pu = RING(t - 2, rs)[0].y;
          }
          const float np = fmaf(-h2x * kb.x, fmaf(rxy, syv, sxpu.y), pp);
          const float nu = fmaf(-h2x * kb.y, sxpu.x, pu);
          const float nv = fmaf(-h2y * kb.y, syp, pv);
          if (t < T) {
            wp[t][sl] = np;
            wv[t][sl] = nv;
            RING(t, rs)[0] = make_float2(np, nu);
          }
          if (t >= T - 1 && (t == T || !pd.last)) {
            const int rho = s - R * T - R * t;
            if (out_col && rho >= 0 && rho < hs) {
              const int64_t e = (int64_t)(Y0 + rho) * nx + x;
              if (!pd.last) {
                float* o = (t == T) ? outB : outA;
                __stcg(o + e, np);
                __stcg(o + PP + e, nu);
                __stcg(o + 2 * PP + e, nv);
              } else {
                // y_(N-1) = prev, y_N = level T-1 at this row, y_(N+1) = new
                const float cp = wp[T - 1][sl], cv = wv[T - 1][sl], cu = RING(T - 1, rs)[0].y;
                __stcg(outA + e, gragg_avg(pp, cp, np));
                __stcg(outA + PP + e, gragg_avg(pu, cu, nu));
                __stcg(outA + 2 * PP + e, gragg_avg(pv, cv, nv));
              }
            }
          }
        }
      }
      ms0 = ms0 + 1 == M ? 0 : ms0 + 1;
      rs0 = rs0 + 1 == UR ? 0 : rs0 + 1;
      if ((s % kSyncEvery) == kSyncEvery - 1) __syncthreads();
    }
  }
}

template <int R>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_passes(const Params P) {
  extern __shared__ float smem[];
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(P.queue, 1);
    __syncthreads();
    const int i = s_item;
    __syncthreads();
    if (i >= P.n_items) return;
    if (threadIdx.x < kMaxDeps) {
      const int d = P.deps[i * kMaxDeps + threadIdx.x];
      if (d >= 0) {
        long long spins = 0;
        while (ld_acquire(P.done + d) == 0) {
          if (++spins > P.spin_limit) {
            atomicCAS(P.err, 0, (int)GBS_ERR_TIMEOUT);
            break;
          }
          __nanosleep(100);
        }
      }
    }
    __syncthreads();
    const Item it = P.items[i];
    const ProbDev& q = P.probs[it.prob];
    const PassDesc pd = P.pdesc[(q.slot * GBS_MAX_SEQ + it.seq) * kMaxPasses + it.pass];
    if (pd.T == 2) run_item<R, 2>(P, it, pd, smem);
#if GBS_FUSED_TMAX >= 6
    else if (pd.T == 6) run_item<R, 6>(P, it, pd, smem);
#endif
#if GBS_FUSED_TMAX >= 8
    else if (pd.T == 8) run_item<R, 8>(P, it, pd, smem);
#endif
    else run_item<R, 4>(P, it, pd, smem);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      st_release(P.done + i, 1);
    }
  }
}

// y_out = sum_k c_k y*_k (per problem, its slot's weights), accumulated in FP32 pairs:
// c_k = chi + clo, the product chi*y is split exactly by one FMA (TwoProd), clo*y is added
// to its error, and the running sum is kept as (hi, lo) with TwoSum.  The accumulated
// error is about 2^-48 of sum_k |c_k y*_k| -- FP64-class -- while using only FP32 units
// (GB300 runs FP64 at a small fraction of the FP32 rate; a plain FP64 sum of 11 terms
// per element would saturate that pipe).
__global__ void k_combine(const ProbDev* probs, int batch, const SlotDev* slots, const float* __restrict__ ystar,
                          int64_t E, float* __restrict__ y_out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = batch - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (probs[mid].state_off <= e) lo = mid;
      else hi = mid - 1;
    }
    const SlotDev& s = slots[probs[lo].slot];
    float sh = 0.f, sl = 0.f;
    for (int k = 0; k < s.m; ++k) {
      const float y = __ldcg(ystar + (int64_t)k * E + e);
      // _rn intrinsics keep the compiler from contracting these into FMAs
      const float p = __fmul_rn(s.chi[k], y);
      const float pe = fmaf(s.clo[k], y, fmaf(s.chi[k], y, -p));   // chi*y - p exactly, plus clo*y
      const float t = __fadd_rn(sh, p);
      const float bv = __fsub_rn(t, sh);
      const float te = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bv)), __fsub_rn(p, bv));
      sl = __fadd_rn(sl, __fadd_rn(te, pe));
      sh = __fadd_rn(t, sl);
      sl = __fsub_rn(sl, __fsub_rn(sh, t));
    }
    y_out[e] = sh + sl;
  }
}

size_t ring_bytes(int R) {
  const int ur = 2 * R + kSyncEvery, m = R * kTMax + kSyncEvery + 1;
  return (size_t)(kTMax * ur + m) * kRow * sizeof(float2);
}

}  // namespace fused

// ===========================================================================
// Host side
// ===========================================================================

struct FusedWork {
  int64_t E = 0;
  int m_max = 0;
  int n_items = 0;
  int grid = 0;
  int R = 0;
  int hseg = 512;
  float* lev = nullptr;
  float* ystar = nullptr;
  fused::Item* items = nullptr;
  int* deps = nullptr;
  int* done = nullptr;   // n_items flags followed by the queue counter
  fused::PassDesc* pdesc = nullptr;
  fused::TileGeo* tgeo = nullptr;
  size_t lev_cap = 0, ystar_cap = 0, items_cap = 0;
  double alg_bytes = 0;   // algorithmic bytes of one k_passes launch
  long long spin_limit = fused::kSpinLimit;
  int inject_wait = 0;    // test hook: item 0 also waits on a flag that nothing sets
};

namespace {

void free_work(FusedWork* w) {
  void* ptrs[] = {w->lev, w->ystar, w->items, w->deps, w->done, w->pdesc, w->tgeo};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  w->lev = w->ystar = nullptr;
  w->items = nullptr;
  w->deps = w->done = nullptr;
  w->pdesc = nullptr;
  w->tgeo = nullptr;
  w->lev_cap = w->ystar_cap = w->items_cap = 0;
}

// Leap-frog levels of sequence N split into passes: first N mod 8 (if nonzero), then 8s.
std::vector<int> pass_plan(int N) {
  std::vector<int> v;
  int rem = N % fused::kTMax;
  if (rem) v.push_back(rem);
  for (int l = rem; l < N; l += fused::kTMax) v.push_back(fused::kTMax);
  return v;
}

fused::TileGeo tiles_of(int nx, int ny, int hseg, int halo) {
  fused::TileGeo g;
  std::memset(&g, 0, sizeof g);
  const int wmax = fused::kThreads - 2 * halo;   // output columns a CTA can hold with its halo
  g.nst = (nx + wmax - 1) / wmax;
  g.nseg = std::max(1, std::min((ny + hseg - 1) / hseg, ny / halo));
  return g;
}

}  // namespace

bool fused_supported(const StepPlan& p, const ProbDev* probs_h) {
  if (p.system != GBS_ACOUSTIC || p.ndim != 2 || p.f64 || (p.R != 2 && p.R != 3)) return false;
  const int halo = p.R * fused::kTMax;
  for (int q = 0; q < p.batch; ++q) {
    // rows wrap at most twice around the period; several strips must each be wider than
    // the halo
    if (probs_h[q].n[1] < halo) return false;
    const fused::TileGeo g = tiles_of(probs_h[q].n[0], probs_h[q].n[1], 512, halo);
    if (g.nst > 1 && probs_h[q].n[0] / g.nst < halo) return false;
  }
  return true;
}

FusedWork* fused_create() { return new FusedWork(); }

void fused_set_test_hooks(FusedWork* w, long long spin_limit, int inject_wait) {
  w->spin_limit = spin_limit;
  w->inject_wait = inject_wait;
}

void fused_destroy(FusedWork* w) {
  if (!w) return;
  free_work(w);
  delete w;
}

template <class T>
static int grow(T** p, size_t* cap, size_t bytes) {
  if (*cap >= bytes) return 0;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMalloc(reinterpret_cast<void**>(p), bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return -1;
  }
  *cap = bytes;
  return 0;
}

int fused_prepare(FusedWork* w, const StepPlan& p, const ProbDev* probs_h, const SlotDev* slots_h, int hseg,
                  char* msg, size_t msglen) {
  using namespace fused;
  w->E = p.state_elems;
  w->R = p.R;
  w->hseg = hseg;
  w->m_max = p.max_m;
  // pass descriptors per (slot, seq, pass)
  std::vector<PassDesc> pdesc((size_t)GBS_MAX_SLOTS * GBS_MAX_SEQ * kMaxPasses);
  std::memset(pdesc.data(), 0, pdesc.size() * sizeof(PassDesc));
  for (int sl = 0; sl < GBS_MAX_SLOTS; ++sl)
    for (int k = 0; k < slots_h[sl].m; ++k) {
      const std::vector<int> pl = pass_plan(slots_h[sl].steps[k]);
      for (size_t qq = 0; qq < pl.size(); ++qq) {
        PassDesc& d = pdesc[((size_t)sl * GBS_MAX_SEQ + k) * kMaxPasses + qq];
        d.T = pl[qq];
        d.first = qq == 0;
        d.last = qq + 1 == pl.size();
      }
    }
  // items, ordered by remaining depth (longest chains first), then problem, sequence, tile
  std::vector<TileGeo> tg(p.batch);
  struct Key {
    int depth, prob, seq, pass, tile;
  };
  std::vector<Key> keys;
  for (int q = 0; q < p.batch; ++q) {
    tg[q] = tiles_of(probs_h[q].n[0], probs_h[q].n[1], hseg, p.R * kTMax);
    const SlotDev& s = slots_h[probs_h[q].slot];
    for (int k = 0; k < s.m; ++k) {
      const int np = (int)pass_plan(s.steps[k]).size();
      for (int qq = 0; qq < np; ++qq)
        for (int t = 0; t < tg[q].nst * tg[q].nseg; ++t) keys.push_back({np - qq, q, k, qq, t});
    }
  }
  std::stable_sort(keys.begin(), keys.end(), [](const Key& a, const Key& b) {
    if (a.depth != b.depth) return a.depth > b.depth;
    if (a.pass != b.pass) return a.pass < b.pass;
    return false;
  });
  const int n = (int)keys.size();
  std::vector<Item> items(n);
  std::vector<int> index_of;  // (prob, seq, pass, tile) -> item index via map
  // flat lookup: offsets per (prob, seq, pass)
  std::vector<int64_t> base((size_t)p.batch * GBS_MAX_SEQ * kMaxPasses, -1);
  {
    int64_t off = 0;
    for (int q = 0; q < p.batch; ++q) {
      const SlotDev& s = slots_h[probs_h[q].slot];
      for (int k = 0; k < s.m; ++k) {
        const int np = (int)pass_plan(s.steps[k]).size();
        for (int qq = 0; qq < np; ++qq) {
          base[((size_t)q * GBS_MAX_SEQ + k) * kMaxPasses + qq] = off;
          off += tg[q].nst * tg[q].nseg;
        }
      }
    }
    index_of.assign((size_t)off, -1);
  }
  for (int i = 0; i < n; ++i) {
    items[i] = {keys[i].prob, keys[i].seq, keys[i].pass, keys[i].tile};
    index_of[base[((size_t)keys[i].prob * GBS_MAX_SEQ + keys[i].seq) * kMaxPasses + keys[i].pass] + keys[i].tile] = i;
  }
  std::vector<int> deps((size_t)n * kMaxDeps, -1);
  for (int i = 0; i < n; ++i) {
    const Item& it = items[i];
    if (it.pass == 0) continue;
    const TileGeo& g = tg[it.prob];
    const int sx = it.tile % g.nst, sy = it.tile / g.nst;
    int nd = 0;
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int tx = ((sx + dx) % g.nst + g.nst) % g.nst, ty = ((sy + dy) % g.nseg + g.nseg) % g.nseg;
        const int j = index_of[base[((size_t)it.prob * GBS_MAX_SEQ + it.seq) * kMaxPasses + it.pass - 1] +
                               ty * g.nst + tx];
        bool dup = false;
        for (int e = 0; e < nd; ++e) dup |= deps[(size_t)i * kMaxDeps + e] == j;
        if (!dup) deps[(size_t)i * kMaxDeps + nd++] = j;
        if (j >= i) {
          std::snprintf(msg, msglen, "fused schedule is not topologically ordered");
          return -1;
        }
      }
  }
  // device buffers
  const size_t lev_bytes = (size_t)4 * p.max_m * p.state_elems * sizeof(float);
  const size_t ys_bytes = (size_t)p.max_m * p.state_elems * sizeof(float);
  if (grow(&w->lev, &w->lev_cap, lev_bytes) || grow(&w->ystar, &w->ystar_cap, ys_bytes)) {
    std::snprintf(msg, msglen, "cudaMalloc of the fused level store (%zu bytes) failed", lev_bytes + ys_bytes);
    return -2;
  }
  if (w->items) cudaFree(w->items);
  if (w->deps) cudaFree(w->deps);
  if (w->done) cudaFree(w->done);
  if (w->pdesc) cudaFree(w->pdesc);
  if (w->tgeo) cudaFree(w->tgeo);
  w->items = nullptr;
  w->deps = w->done = nullptr;
  w->pdesc = nullptr;
  w->tgeo = nullptr;
  if (cudaMalloc(&w->items, sizeof(Item) * std::max(n, 1)) != cudaSuccess ||
      cudaMalloc(&w->deps, sizeof(int) * kMaxDeps * std::max(n, 1)) != cudaSuccess ||
      cudaMalloc(&w->done, sizeof(int) * (n + 2)) != cudaSuccess ||
      cudaMalloc(&w->pdesc, sizeof(PassDesc) * pdesc.size()) != cudaSuccess ||
      cudaMalloc(&w->tgeo, sizeof(TileGeo) * p.batch) != cudaSuccess) {
    cudaGetLastError();
    std::snprintf(msg, msglen, "cudaMalloc of the fused schedule failed");
    return -2;
  }
  // optional failure-detection hook: item 0 depends on flag n + 1, which no item ever sets
  if (w->inject_wait && n > 0) deps[kMaxDeps - 1] = n + 1;
  if (cudaMemcpy(w->items, items.data(), sizeof(Item) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(w->deps, deps.data(), sizeof(int) * deps.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(w->pdesc, pdesc.data(), sizeof(PassDesc) * pdesc.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(w->tgeo, tg.data(), sizeof(TileGeo) * p.batch, cudaMemcpyHostToDevice) != cudaSuccess) {
    std::snprintf(msg, msglen, "upload of the fused schedule failed");
    return -3;
  }
  w->n_items = n;
  // algorithmic bytes per launch: every item reads its two input levels (y_0 and f0 for a
  // first pass) and the two media over its tile once and writes two levels (one average)
  {
    double by = 0;
    for (int i = 0; i < n; ++i) {
      const Item& it = items[i];
      const TileGeo& g = tg[it.prob];
      const int sx = it.tile % g.nst, sy = it.tile / g.nst;
      const int nx = probs_h[it.prob].n[0], ny = probs_h[it.prob].n[1];
      const double pts = (double)(((sx + 1) * nx) / g.nst - (sx * nx) / g.nst) *
                         (((sy + 1) * ny) / g.nseg - (sy * ny) / g.nseg);
      const PassDesc& d = pdesc[((size_t)probs_h[it.prob].slot * GBS_MAX_SEQ + it.seq) * kMaxPasses + it.pass];
      by += pts * 4.0 * (2.0 * p.F + 2.0 + (d.last ? 1.0 : 2.0) * p.F);
    }
    w->alg_bytes = by;
  }
  // persistent grid: resident CTAs per SM times SMs
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = ring_bytes(p.R);
  if (p.R == 2) {
    cudaFuncSetAttribute(k_passes<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_passes<2>, kThreads, smem);
  } else {
    cudaFuncSetAttribute(k_passes<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_passes<3>, kThreads, smem);
  }
  if (cudaGetLastError() != cudaSuccess || per_sm < 1) {
    std::snprintf(msg, msglen, "the fused kernel cannot be resident (smem %zu bytes)", smem);
    return -3;
  }
  w->grid = std::max(1, std::min(n, sms * per_sm));
  return 0;
}

int fused_macro_step(FusedWork* w, const StepPlan& p, const void* y_in, void* y_out, cudaStream_t s, int* err) {
  using namespace fused;
  int launches = 0;
  if (launch_f0(p, y_in, s) < 0) return -1;
  ++launches;
  if (cudaMemsetAsync(w->done, 0, sizeof(int) * (w->n_items + 2), s) != cudaSuccess) return -1;
  Params P;
  P.items = w->items;
  P.deps = w->deps;
  P.n_items = w->n_items;
  P.done = w->done;
  P.queue = w->done + w->n_items;
  P.err = err;
  P.probs = p.probs;
  P.slots = p.slots;
  P.hk = p.hk;
  P.hkf = p.hkf;
  P.kappa = static_cast<const float*>(p.kappa);
  P.b = static_cast<const float*>(p.b);
  P.y0 = static_cast<const float*>(y_in);
  P.f0 = static_cast<const float*>(p.f0);
  P.lev = w->lev;
  P.ystar = w->ystar;
  P.E = w->E;
  P.pdesc = w->pdesc;
  P.tgeo = w->tgeo;
  P.spin_limit = w->spin_limit;
  const size_t smem = ring_bytes(w->R);
  const int u = timing_begin(p, s);
  if (w->R == 2) k_passes<2><<<w->grid, kThreads, smem, s>>>(P);
  else k_passes<3><<<w->grid, kThreads, smem, s>>>(P);
  timing_end(p, u, s, w->alg_bytes);
  ++launches;
  k_combine<<<1024, 256, 0, s>>>(p.probs, p.batch, p.slots, w->ystar, w->E, static_cast<float*>(y_out));
  ++launches;
  if (cudaPeekAtLastError() != cudaSuccess) return -1;
  return launches;
}

}  // namespace gbs
