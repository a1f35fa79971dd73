// Time-blocked FP32 macro-step for 2D acoustics: a persistent dataflow kernel.
//
// One macro-step (Sec. 2.1 eq. "GBS", Sec. 3.6, Sec. 3.2) runs as
//   1. f0 = f(y_in)              point-parallel, shared by every sequence (Sec. 3.6); the same
//                                kernel interleaves the media (FP32 pairs: a prologue converts
//                                y_in and the media and evaluates f0 in pairs)
//   2. k_passes                  all Forward-Euler / leap-frog levels of all sequences
//   3. k_combine                 y_out = sum_k c_k y*_k: in FP64 (FP32 states: y_0 + sum_k c_k d*_k,
//                                the increment form), or in compensated FP32 pairs
//
// Work items.  Sequence k has the Forward-Euler level y_1 and N_k leap-frog
// levels y_2 .. y_(N+1).  The leap-frog levels are cut into passes of T <= kTMax
// levels (the first pass takes N mod kTMax), and every pass into tiles: strips of
// at most kThreads - 2 R kTMax columns times segments of rows.  An item (problem,
// k, pass, tile) reads the two levels (y_(n-1), y_n) of the previous pass over
// its tile plus an R*T halo, advances them T levels and writes (y_(n+T-1),
// y_(n+T)) -- or, in the sequence's last pass, the average
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
// s - R T - R t.  Every level keeps the last 2R+1 rows of (p, v) of its
// thread's column in registers (the y-stencils and the leap-frog "previous"
// value) and publishes its newest (p, u) row in shared memory, from which the
// neighbouring columns take their x-stencils.  Stencil sums use packed FP32-pair
// arithmetic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "gbs_ds.cuh"
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
  const float4* hkq;     // FP32: split step constants per problem x sequence (fp32_step_consts)
  const float4* aux;     // FP32: per point (kappa, b, f0_p, f0_u), written by the f0 kernel
  const float* init;     // [2][E]: y_0, f0
  float* lev;            // [seq][set][2][E]
  float* ystar;          // [seq][E]
  int64_t E;
  const PassDesc* pdesc; // [slot][seq][pass]
  const TileGeo* tgeo;   // per problem
  long long spin_limit;  // polls of a dependency flag before GBS_ERR_TIMEOUT
  // GBS_F32X2: init, lev and ystar hold (hi, lo) float pairs (8 bytes per element); the media
  // as pairs
  const dsf* kap2;
  const dsf* b2;
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

// Tensor memory (TMEM) as per-thread scratch for the FP32 sweep's forcing ring (below).  A CTA
// allocates kTmemCols columns of the SM's 512 x 128-lane TMEM; warp w reaches only lanes
// 32 (w mod 4) .. 32 (w mod 4) + 31, so warps w and w + 4 take different halves of the columns.
// Thread t of a warp reads and writes its own lane with the 32x32b shape.  Two CTAs per SM use
// 2 kTmemCols <= 512 columns, so an allocation never waits.
constexpr int kTmemCols = 256;
constexpr int kGSlots = 16;   // ring of per-row constants (power of two > R T), 8 words per row
// No "memory" clobbers: these touch only tensor memory, and volatile asm statements keep their
// order among themselves; a clobber would also pin every global and shared access around them.
// A load's registers are valid only after tmem_wait_ld8, which takes them as read-write operands
// so that no use is scheduled before it.
__device__ __forceinline__ void tmem_st8(uint32_t ta, float a, float b, float c, float d, float e, float f, float g,
                                         float h) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(ta),
               "r"(__float_as_uint(a)), "r"(__float_as_uint(b)), "r"(__float_as_uint(c)), "r"(__float_as_uint(d)),
               "r"(__float_as_uint(e)), "r"(__float_as_uint(f)), "r"(__float_as_uint(g)), "r"(__float_as_uint(h)));
}
struct Row8 {
  uint32_t v[8];
};
__device__ __forceinline__ void tmem_ld8(uint32_t ta, Row8& r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r.v[0]), "=r"(r.v[1]), "=r"(r.v[2]), "=r"(r.v[3]), "=r"(r.v[4]), "=r"(r.v[5]), "=r"(r.v[6]),
                 "=r"(r.v[7])
               : "r"(ta));
}
__device__ __forceinline__ void tmem_wait_ld8(Row8& r) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r.v[0]), "+r"(r.v[1]), "+r"(r.v[2]), "+r"(r.v[3]), "+r"(r.v[4]), "+r"(r.v[5]), "+r"(r.v[6]),
                 "+r"(r.v[7]));
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;"); }

// Shared memory of one CTA (float2 words):
//   level planes  [kTMax][U][kRow]        (p, u) of the newest U = 2R + 1 rows of levels 0..T-1,
//                                          rows padded by kPad so every x-stencil stays inside
//   (FP32 pairs also:) media planes [U][kThreads] of float4, the scaled media of a pass's rows
// A row's slot is its local row index mod U, a compile-time constant in a sweep unrolled by U,
// so no ring index is computed at run time.  A level-t row is read by the x-stencils of level
// t+1 R steps after it is written and by its own thread (the leap-frog "previous" u) 2R steps
// after; it is overwritten U = 2R+1 steps after.  A barrier at least every R steps therefore
// orders both the read after the write and the overwrite after the read.  The FP32 sweep keeps
// the per-row constants (scaled media, forcing) in tensor memory instead (run_item).
constexpr int kPad = 4;
constexpr int kRow = kThreads + 2 * kPad;

// finite-difference weights as integers m_j over a common divisor (fd_int / fd_div: 8, -1 over 12;
// 45, -9, 1 over 60), as (m, m) pairs for the packed sums; exact in FP32, the divisor is folded
// into the per-row scaling
template <int R>
__device__ __forceinline__ float2 fdc(int j) { return make_float2(fd_int<R>(j), fd_int<R>(j)); }

// packed FP32 pairs (Blackwell f32x2 instructions): a - b, c * d + e, c * d
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
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

// x-derivative sums of (p, u) over a level-plane row, unscaled: sum_j m_j (row[+j] - row[-j]),
// the difference taken first (exact for smooth fields) and weighted in pairs
template <int R>
__device__ __forceinline__ float2 xsum2(const float2* row) {
  float2 acc = __fmul2_rn(fdc<R>(1), f2sub(row[1], row[-1]));
#pragma unroll
  for (int j = 2; j <= R; ++j) acc = __ffma2_rn(fdc<R>(j), f2sub(row[j], row[-j]), acc);
  return acc;
}

// y-derivative sums of (p, v) over a register window indexed by row mod U, unscaled
template <int R>
__device__ __forceinline__ float2 ysum2(const float2 (&w)[2 * R + 1], int r) {
  constexpr int U = 2 * R + 1;
  float2 acc = __fmul2_rn(fdc<R>(1), f2sub(w[(r + 1) % U], w[(r + U - 1) % U]));
#pragma unroll
  for (int j = 2; j <= R; ++j) acc = __ffma2_rn(fdc<R>(j), f2sub(w[(r + j) % U], w[(r + U - j) % U]), acc);
  return acc;
}

// The FP32 sweep runs in increment form (gbs_stencil.cuh): the levels hold d_n = y_n - y_0, the
// first pass starts from (d_0, d_1) = (0, h f0), and every leap-frog update adds the forcing
// g = 2h f0 of its row.  The stencil sums use integer weights; their divisor, 1 / dx and -2h
// form one constant s2, and the scaled media s2 kappa and s2 b are kept as float pairs (hi +
// lo, about 2^-48 relative), so that no rounding of the scaling is shared by the points and
// steps of a sequence (that would perturb its operator coherently, which the combine's weights
// and the modes near the stability limit amplify).  When level 0 reaches a row it computes the
// row's eight constants (s2 kappa and s2 b as hi and lo pairs, g for p, v and u), which the T levels that pass over the
// row later read from a ring of kGSlots rows per thread in tensor memory (tbase: this thread's
// lane and column base): row r's slot is r mod kGSlots, and a row is needed for R T < kGSlots
// steps.  A slot written at step s is read from step s + R on; every R steps the sweep waits
// for its tensor-memory stores to complete before its barrier, so each read sees them.
template <int R, int T>
__device__ __forceinline__ void run_item(const Params& P, const Item& it, const PassDesc& pd, float2* smem,
                                         uint32_t tbase) {
  constexpr int U = 2 * R + 1;       // window rows = plane slots
  constexpr int OFF = 64 * U;        // keeps compile-time slot arithmetic non-negative
  const int tid = threadIdx.x;
  const ProbDev q = P.probs[it.prob];
  const TileGeo tg = P.tgeo[it.prob];
  const int nx = q.n[0], ny = q.n[1];
  const int PPn = nx * ny;           // points per field (< 2^31, checked at creation)
  const int sx = it.tile % tg.nst, sy = it.tile / tg.nst;
  const int x0 = (sx * nx) / tg.nst;
  const int wout = ((sx + 1) * nx) / tg.nst - x0;
  const int Y0 = (sy * ny) / tg.nseg;
  const int hs = ((sy + 1) * ny) / tg.nseg - Y0;
  const int x = wrapi(x0 - R * T + tid, nx);
  const float4 hq = P.hkq[it.prob * GBS_MAX_SEQ + it.seq];
  const float gh = hq.x, gl = hq.y;                        // 2h as a float pair
  const float sh2 = -hq.z, sl2 = -hq.w;                    // s2 = -2h / (div dx) as a float pair
  const float rxy = q.rr[1];                               // y-stencil weight relative to x (dx / dy)
  const float4* auxm = P.aux + q.media_off;               // (kappa, b, f0_p, f0_u) per point
  const float* f0v = P.init + P.E + q.state_off + 2 * (int64_t)PPn;   // f0_v
  // the two input levels (d_(n-1), d_n) are E apart (a first pass reads only f0: d_0 = 0,
  // d_1 = h f0), and so are the two output levels (or the average)
  const float* inA = pd.first ? P.init + q.state_off
                              : P.lev + ((int64_t)(it.seq * 2 + ((it.pass - 1) & 1)) * 2) * P.E + q.state_off;
  float* outA = pd.last ? P.ystar + (int64_t)it.seq * P.E + q.state_off
                        : P.lev + ((int64_t)(it.seq * 2 + (it.pass & 1)) * 2) * P.E + q.state_off;
  const int64_t E = P.E;
  const bool out_col = tid >= R * T && tid < R * T + wout;
  float2* const lvl = smem + kPad + tid;                                  // plane t, slot r: lvl[(t U + r) kRow]

  // (p, v) windows of levels 0..T-1.  Level t computes local row s - R T - R t at sweep step
  // s.  Rows before a level's first valid row (s < 2 R t) are computed from not-yet-valid
  // inputs and never reach a valid row: valid level-t rows start at -R (T - t) and read level
  // t-1 rows from -R (T - t) - R on, which are valid.  So no step is guarded.
  float2 w[T][U];
#pragma unroll
  for (int t = 0; t < T; ++t)
#pragma unroll
    for (int u = 0; u < U; ++u) w[t][u] = make_float2(0.f, 0.f);

  const int S = hs + 2 * R * T;
  int e0 = wrapf(Y0 - R * T, ny) * nx + x;       // level 0's row at step 0
  int e1 = wrapf(Y0 - R * T - R, ny) * nx + x;   // level -1 at level 1's row at step 0
  int eo = (Y0 - 2 * R * T) * nx + x;            // level T's output row at step 0 (unwrapped)
  // raw loads of the next step (consumed at the next step's commit): the media and f0 at level
  // 0's row (f0 gives the forcing, and in a first pass level 0 = h f0), and in later passes
  // level 0 and level -1 (at level 1's row; in a first pass d_0 = 0)
  float n0p = 0.f, n0u = 0.f, n0v = 0.f, nfv, n1p = 0.f, n1u = 0.f, n1v = 0.f;
  float4 na;
  auto fetch = [&]() {
    na = __ldg(auxm + e0);
    nfv = __ldg(f0v + e0);
    if (!pd.first) {
      const float* a = inA + e1;
      const float* b = inA + E + e0;
      n0p = __ldcg(b);
      n0u = __ldcg(b + PPn);
      n0v = __ldcg(b + 2 * PPn);
      n1p = __ldcg(a);
      n1u = __ldcg(a + PPn);
      n1v = __ldcg(a + 2 * PPn);
    }
  };
  // L2 prefetch of the rows the next block of U steps loads, so that the one-step-ahead
  // register loads find them in L2: warps 0-2 take level 0's fields, warps 3-5 level -1's (in a
  // first pass the same y_0 rows, R behind, that level 0 also reads).  A sample every 128
  // bytes of the CTA's 256-column row segment touches each of its lines.  The media (a fifth
  // of the bytes, small enough to stay in L2 across sequences) are not prefetched; measured,
  // prefetching them or R more rows of level -1 was slower, and so were bulk range prefetches.
  const int xf = wrapi(x0 - R * T, nx);   // column of thread 0
  auto prefetch_block = [&](int sn) {
    const int wq = tid >> 5;
    if (wq > 5 || pd.first) return;   // warps 6 and 7 issue none, nor any warp in a first pass
    const int row0 = wrapi(Y0 - R * T + sn - (wq >= 3 ? R : 0), ny);
    const float* base = wq < 3 ? inA + E + wq * PPn : inA + (wq - 3) * PPn;
    constexpr int kSamp = 9;   // columns 32 floats (one line) apart, plus the last one
    for (int i = tid & 31; i < U * kSamp; i += 32) {
      const int j = i / kSamp, c = i - j * kSamp;
      int row = row0 + j;
      if (row >= ny) row -= ny;
      const int col = (xf + (c + 1 < kSamp ? c * 32 : kThreads - 1)) % nx;
      asm volatile("prefetch.global.L2 [%0];" ::"l"(base + (size_t)row * nx + col));
    }
  };
  fetch();
  for (int sb = 0; sb < S; sb += U) {
    prefetch_block(sb + U);
#pragma unroll
    for (int uu = 0; uu < U; ++uu) {
      const int s = sb + uu;
      if (s >= S) break;
      // ---- level 0 (local row s - R T), the row's constants, level -1 ----
      const int r0 = (uu + OFF - R * T) % U;
      float p0 = n0p, u0 = n0u, v0 = n0v;
      // the forcing g = 2h f0 (packed for (p, v)); in a first pass level 0 is d_1 = h f0 = g / 2
      const float2 gpv = mul_split2(make_float2(gh, gh), make_float2(gl, gl), make_float2(na.z, nfv));
      const float gu = mul_split(gh, gl, na.w);
      if (pd.first) {
        p0 = 0.5f * gpv.x;
        u0 = 0.5f * gu;
        v0 = 0.5f * gpv.y;
      }
      {
        // (s2 kappa, s2 b) as pairs: the rounded products, then their exact errors plus the lo parts
        const float2 m = make_float2(na.x, na.y), shv = make_float2(sh2, sh2);
        const float2 kbh = __fmul2_rn(shv, m);
        const float2 kbl = __ffma2_rn(make_float2(sl2, sl2), m, __ffma2_rn(shv, m, make_float2(-kbh.x, -kbh.y)));
        tmem_st8(tbase + 8u * ((uint32_t)(sb + uu + 64 * kGSlots - R * T) & (kGSlots - 1)), kbh.x, kbh.y, kbl.x,
                 kbl.y, gpv.x, gpv.y, gu, 0.f);
      }
      w[0][r0] = make_float2(p0, v0);
      lvl[r0 * kRow] = make_float2(p0, u0);
      const float2 am_pv = make_float2(n1p, n1v);
      const float am_u = n1u;
      // ---- prefetch step s + 1 (rows wrap, so the extra fetch after the last step is in bounds) ----
      e0 += nx;
      if (e0 >= PPn) e0 -= PPn;
      e1 += nx;
      if (e1 >= PPn) e1 -= PPn;
      fetch();
      const bool stT = out_col && (unsigned)(s - 2 * R * T) < (unsigned)hs;
      const bool stT1 = out_col && (unsigned)(s - 2 * R * T + R) < (unsigned)hs;
      // ---- levels 1..T ----
#pragma unroll
      for (int t = 1; t <= T; ++t) {
        const int r = (uu + OFF - R * T - R * t) % U;   // slot of this level's row
        Row8 rc;   // this row's constants, loaded while the stencil sums run
        tmem_ld8(tbase + 8u * ((uint32_t)(sb + uu + 64 * kGSlots - R * T - R * t) & (kGSlots - 1)), rc);
        const float2 sxv = xsum2<R>(lvl + ((t - 1) * U + r) * kRow);   // (sum_x p, sum_x u)
        const float2 syv = ysum2<R>(w[t - 1], r);                       // (sum_y p, sum_y v)
        float2 ppv;
        float pu;
        if (t == 1) {
          ppv = am_pv;
          pu = am_u;
        } else {
          ppv = w[t - 2][r];
          pu = lvl[((t - 2) * U + r) * kRow].y;
        }
        tmem_wait_ld8(rc);
        const float2 kbh = make_float2(__uint_as_float(rc.v[0]), __uint_as_float(rc.v[1]));   // (s2 kappa, s2 b) hi
        const float2 kbl = make_float2(__uint_as_float(rc.v[2]), __uint_as_float(rc.v[3]));   // and lo
        const float2 gpv = make_float2(__uint_as_float(rc.v[4]), __uint_as_float(rc.v[5]));   // forcing of (p, v)
        // d_(n+1) = d_(n-1) + g + s2 (kappa (sum_x u + rxy sum_y v), b sum_x p, b rxy sum_y p), with
        // (p, v) as one packed lane pair: sums (sum_x u + rxy sum_y v, rxy sum_y p)
        const float2 spv = __ffma2_rn(make_float2(rxy, rxy), make_float2(syv.y, syv.x), make_float2(sxv.y, 0.f));
        const float2 npv = __ffma2_rn(kbh, spv, __ffma2_rn(kbl, spv, __fadd2_rn(ppv, gpv)));
        const float np = npv.x, nv = npv.y;
        const float nu = fmaf(kbh.y, sxv.x, fmaf(kbl.y, sxv.x, pu + __uint_as_float(rc.v[6])));
        if (t < T) {
          w[t][r] = make_float2(np, nv);
          lvl[(t * U + r) * kRow] = make_float2(np, nu);
        }
        if (!pd.last) {
          if (t == T - 1 && stT1) {
            float* o = outA + (eo + R * nx);
            __stcs(o, np);
            __stcs(o + PPn, nu);
            __stcs(o + 2 * PPn, nv);
          }
          if (t == T && stT) {
            float* o = outA + E + eo;
            __stcs(o, np);
            __stcs(o + PPn, nu);
            __stcs(o + 2 * PPn, nv);
          }
        } else if (t == T && stT) {
          // y_(N-1) = previous, y_N = level T-1 at this row, y_(N+1) = new
          const float2 cpv = w[T - 1][r];
          const float cu = lvl[((T - 1) * U + r) * kRow].y;
          float* o = outA + eo;
          __stcs(o, gragg_avg(ppv.x, cpv.x, np));
          __stcs(o + PPn, gragg_avg(pu, cu, nu));
          __stcs(o + 2 * PPn, gragg_avg(ppv.y, cpv.y, nv));
        }
      }
      eo += nx;
      if (uu % R == R - 1 || uu == U - 1) {
        tmem_wait_st();
        __syncthreads();
      }
    }
  }
}

// ---------------------------------------------------------------------------
// The same sweep in FP32-pair arithmetic (GBS_F32X2: FP64 states carried as hi + lo float pairs),
// passes of two levels.  Every value is a pair: (p, v) windows as ds2 (two pairs per packed
// lane), (p, u) plane entries as float4 (p.hi, u.hi, p.lo, u.lo), the scaled media as float4
// (kappa'.hi, kappa'.lo, b'.hi, b'.lo); the stencil sums are exact integer-weight pair sums
// (isum_x2, their divisor folded into the media scaling) and every other sum, product and update
// is a pair operation (gbs_ds.cuh).  With T = 2 the register windows and shared planes take the
// room the FP32 sweep takes at T = 4.
// ---------------------------------------------------------------------------
constexpr int kTX2 = 2;

// x-sums of (p, u) and y-sums of (p, v) in the integer form (times fd_div)
template <int R>
__device__ __forceinline__ ds2 xsum_x2i(const float4* row) {
  return isum_x2<R>([&](int j) { const float4 v = row[j]; return make_float2(v.x, v.y); },
                    [&](int j) { const float4 v = row[j]; return make_float2(v.z, v.w); });
}
template <int R>
__device__ __forceinline__ ds2 ysum_x2i(const ds2 (&w)[2 * R + 1], int r) {
  constexpr int U = 2 * R + 1;
  return isum_x2<R>([&](int j) { return w[(r + j + U) % U].hi; }, [&](int j) { return w[(r + j + U) % U].lo; });
}

__device__ __forceinline__ dsf ds_of(float2 a) { return dsf(a.x, a.y); }
__device__ __forceinline__ float2 f2_of(dsf a) { return make_float2(a.hi, a.lo); }

template <int R>
__device__ __forceinline__ void run_item_x2(const Params& P, const Item& it, const PassDesc& pd, float4* smem) {
  constexpr int T = kTX2;
  constexpr int U = 2 * R + 1;
  constexpr int OFF = 64 * U;
  const int tid = threadIdx.x;
  const ProbDev q = P.probs[it.prob];
  const TileGeo tg = P.tgeo[it.prob];
  const int nx = q.n[0], ny = q.n[1];
  const int PPn = nx * ny;
  const int sx = it.tile % tg.nst, sy = it.tile / tg.nst;
  const int x0 = (sx * nx) / tg.nst;
  const int wout = ((sx + 1) * nx) / tg.nst - x0;
  const int Y0 = (sy * ny) / tg.nseg;
  const int hs = ((sy + 1) * ny) / tg.nseg - Y0;
  const int x = wrapi(x0 - R * T + tid, nx);
  const double hd = P.hk[it.prob * GBS_MAX_SEQ + it.seq];
  const dsf h1 = dsf(hd);
  const dsf mh = dsf(-2.0 * hd * q.inv_dx[0] / fd_div<R>());        // -2h / (dx div): integer-weight sums
  const double rxyd = q.inv_dx[1] / q.inv_dx[0];
  const bool unit = rxyd == 1.0;
  const dsf rxy = dsf(rxyd);
  const dsf* kap = P.kap2 + q.media_off;
  const dsf* bmd = P.b2 + q.media_off;
  const float2* init = reinterpret_cast<const float2*>(P.init);
  float2* lev = reinterpret_cast<float2*>(P.lev);
  float2* ystar = reinterpret_cast<float2*>(P.ystar);
  const int64_t E = P.E;
  const float2* inA = pd.first ? init + q.state_off : lev + ((int64_t)(it.seq * 2 + ((it.pass - 1) & 1)) * 2) * E + q.state_off;
  float2* outA = pd.last ? ystar + (int64_t)it.seq * E + q.state_off
                         : lev + ((int64_t)(it.seq * 2 + (it.pass & 1)) * 2) * E + q.state_off;
  const bool out_col = tid >= R * T && tid < R * T + wout;
  float4* const lvl = smem + kPad + tid;                // plane t, slot r: lvl[(t U + r) kRow]
  float4* const med = smem + T * U * kRow + tid;        // slot r: med[r kThreads]

  ds2 w[T][U];
#pragma unroll
  for (int t = 0; t < T; ++t)
#pragma unroll
    for (int u = 0; u < U; ++u) w[t][u] = ds2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};

  const int S = hs + 2 * R * T;
  int e0 = wrapf(Y0 - R * T, ny) * nx + x;
  int e1 = wrapf(Y0 - R * T - R, ny) * nx + x;
  int eo = (Y0 - 2 * R * T) * nx + x;
  float2 n0[3], y0v[3], n1[3];
  dsf nk, nb;
#pragma unroll
  for (int f = 0; f < 3; ++f) y0v[f] = make_float2(0.f, 0.f);
  auto fetch = [&]() {
#pragma unroll
    for (int f = 0; f < 3; ++f) {
      n0[f] = __ldcg(inA + E + e0 + f * PPn);
      if (pd.first) y0v[f] = __ldcg(inA + e0 + f * PPn);
      n1[f] = __ldcg(inA + e1 + f * PPn);
    }
    nk = ldg(kap + e0);
    nb = ldg(bmd + e0);
  };
  // L2 prefetch of the next block of U rows (as in run_item; a pair row segment is 16 lines)
  const int xf = wrapi(x0 - R * T, nx);
  auto prefetch_block = [&](int sn) {
    const int wq = tid >> 5;
    if (wq > 5) return;
    const int row0 = wrapi(Y0 - R * T + sn - (wq >= 3 ? R : 0), ny);
    const float2* base = wq < 3 ? inA + E + wq * PPn : inA + (wq - 3) * PPn;
    constexpr int kSamp = 17;   // columns 16 pairs (one line) apart, plus the last one
    for (int i = tid & 31; i < U * kSamp; i += 32) {
      const int j = i / kSamp, c = i - j * kSamp;
      int row = row0 + j;
      if (row >= ny) row -= ny;
      const int col = (xf + (c + 1 < kSamp ? c * 16 : kThreads - 1)) % nx;
      asm volatile("prefetch.global.L2 [%0];" ::"l"(base + (size_t)row * nx + col));
    }
  };
  fetch();
  for (int sb = 0; sb < S; sb += U) {
    prefetch_block(sb + U);
#pragma unroll
    for (int uu = 0; uu < U; ++uu) {
      const int s = sb + uu;
      if (s >= S) break;
      // ---- level 0, level -1, media ----
      const int r0 = (uu + OFF - R * T) % U;
      dsf p0 = ds_of(n0[0]), u0 = ds_of(n0[1]), v0 = ds_of(n0[2]);
      if (pd.first) {
        p0 = ds_of(y0v[0]) + h1 * p0;
        u0 = ds_of(y0v[1]) + h1 * u0;
        v0 = ds_of(y0v[2]) + h1 * v0;
      }
      w[0][r0] = make_ds2(p0, v0);
      lvl[r0 * kRow] = make_float4(p0.hi, u0.hi, p0.lo, u0.lo);
      {
        const dsf km = nk * mh, bk = nb * mh;
        med[r0 * kThreads] = make_float4(km.hi, km.lo, bk.hi, bk.lo);
      }
      const ds2 am_pv = make_ds2(ds_of(n1[0]), ds_of(n1[2]));
      const dsf am_u = ds_of(n1[1]);
      e0 += nx;
      if (e0 >= PPn) e0 -= PPn;
      e1 += nx;
      if (e1 >= PPn) e1 -= PPn;
      fetch();
      const bool stT = out_col && (unsigned)(s - 2 * R * T) < (unsigned)hs;
      const bool stT1 = out_col && (unsigned)(s - 2 * R * T + R) < (unsigned)hs;
      // ---- levels 1..T ----
#pragma unroll
      for (int t = 1; t <= T; ++t) {
        const int r = (uu + OFF - R * T - R * t) % U;
        const float4 mf = med[r * kThreads];
        const dsf km(mf.x, mf.y), bk(mf.z, mf.w);
        const ds2 sxv = xsum_x2i<R>(lvl + ((t - 1) * U + r) * kRow);  // div (sum_x p, sum_x u)
        const ds2 syv = ysum_x2i<R>(w[t - 1], r);                      // div (sum_y p, sum_y v)
        ds2 ppv;
        dsf pu;
        if (t == 1) {
          ppv = am_pv;
          pu = am_u;
        } else {
          ppv = w[t - 2][r];
          const float4 o = lvl[((t - 2) * U + r) * kRow];
          pu = dsf(o.y, o.w);
        }
        // (p, v) += (kappa', b') * (sum_x u + rxy sum_y v, rxy sum_y p);  u += b' sum_x p
        const dsf syv_v = unit ? lane_y(syv) : rxy * lane_y(syv);
        const dsf syv_p = unit ? lane_x(syv) : rxy * lane_x(syv);
        const ds2 npv = ppv + ds2_mul(make_ds2(lane_y(sxv) + syv_v, syv_p), make_ds2(km, bk));
        const dsf nu = pu + bk * lane_x(sxv);
        const dsf np = lane_x(npv), nv = lane_y(npv);
        if (t < T) {
          w[t][r] = npv;
          lvl[(t * U + r) * kRow] = make_float4(np.hi, nu.hi, np.lo, nu.lo);
        }
        if (!pd.last) {
          if (t == T - 1 && stT1) {
            float2* o = outA + (eo + R * nx);
            __stcs(o, f2_of(np));
            __stcs(o + PPn, f2_of(nu));
            __stcs(o + 2 * PPn, f2_of(nv));
          }
          if (t == T && stT) {
            float2* o = outA + E + eo;
            __stcs(o, f2_of(np));
            __stcs(o + PPn, f2_of(nu));
            __stcs(o + 2 * PPn, f2_of(nv));
          }
        } else if (t == T && stT) {
          const ds2 cpv = w[T - 1][r];
          const float4 co = lvl[((T - 1) * U + r) * kRow];
          float2* o = outA + eo;
          __stcs(o, f2_of(gragg_avg(lane_x(ppv), lane_x(cpv), np)));
          __stcs(o + PPn, f2_of(gragg_avg(pu, dsf(co.y, co.w), nu)));
          __stcs(o + 2 * PPn, f2_of(gragg_avg(lane_y(ppv), lane_y(cpv), nv)));
        }
      }
      eo += nx;
      if (uu % R == R - 1 || uu == U - 1) __syncthreads();
    }
  }
}

template <int R, bool X2>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_passes(const Params P) {
  extern __shared__ float2 smem[];
  __shared__ int s_item;
  __shared__ uint32_t s_tmem;
  const int warp = threadIdx.x >> 5;
  if constexpr (!X2) {
    // the FP32 sweep's forcing ring lives in tensor memory (run_item)
    if (warp == 0) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                       (uint32_t)__cvta_generic_to_shared(&s_tmem)),
                   "r"(kTmemCols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  const uint32_t tbase = X2 ? 0u : s_tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(kTmemCols / 2) * (warp >> 2);
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(P.queue, 1);
    __syncthreads();
    const int i = s_item;
    __syncthreads();
    if (i >= P.n_items) break;
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
    if constexpr (X2) run_item_x2<R>(P, it, pd, reinterpret_cast<float4*>(smem));
    else if (pd.T == 2) run_item<R, 2>(P, it, pd, smem, tbase);
#if GBS_FUSED_TMAX >= 6
    else if (pd.T == 6) run_item<R, 6>(P, it, pd, smem, tbase);
#endif
#if GBS_FUSED_TMAX >= 8
    else if (pd.T == 8) run_item<R, 8>(P, it, pd, smem, tbase);
#endif
    else run_item<R, 4>(P, it, pd, smem, tbase);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      st_release(P.done + i, 1);
    }
  }
  if constexpr (!X2) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem), "r"(kTmemCols) : "memory");
  }
}

__device__ __forceinline__ int problem_of(const ProbDev* probs, int batch, int64_t e) {
  int lo = 0, hi = batch - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (probs[mid].state_off <= e) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// y_out = y_0 + sum_k c_k d*_k (per problem, its slot's weights): the increment form's combine
// (y*_k = y_0 + d*_k, sum_k c_k = 1; Sec. 2.1, Sec. 3.2), in ascending k.  kF64: the averages and
// y_0 are promoted to FP64 exactly and summed with FP64 FMAs, rounded to FP32 once (GB300's FP64
// pipe makes this the costlier variant); otherwise the sum runs in compensated FP32 pairs
// (pair_combine_add, error about 2^-48 of sum_k |c_k d*_k|, FP32 units only).  Four consecutive
// elements per thread: the loads of all sequences are issued before the sums (float4 when the
// group is 16-byte aligned and inside one problem, else element by element).  y_0 may be y_out
// (in place): each element is read before it is written by the same thread.
template <bool kF64>
__global__ void __launch_bounds__(256) k_combine(const ProbDev* probs, int batch, const SlotDev* slots,
                                                 const float* __restrict__ dstar, int64_t E, const float* y0,
                                                 float* y_out) {
  const int64_t groups = (E + 3) / 4;
  // float4 access needs E % 4 == 0 (sequence blocks and y groups 16-byte aligned; dstar is a
  // library allocation) and 16-byte aligned caller buffers
  const bool vec = (E % 4) == 0 && ((reinterpret_cast<uintptr_t>(y_out) | reinterpret_cast<uintptr_t>(y0)) & 15) == 0;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < groups; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e0 = 4 * g;
    const int q0 = problem_of(probs, batch, e0);
    const int64_t e3 = e0 + 3 < E ? e0 + 3 : E - 1;
    if (vec && (q0 + 1 >= batch || probs[q0 + 1].state_off > e3)) {
      const SlotDev& s = slots[probs[q0].slot];
      float4 d[GBS_MAX_SEQ];
#pragma unroll
      for (int k = 0; k < GBS_MAX_SEQ; ++k)
        if (k < s.m) d[k] = __ldcs(reinterpret_cast<const float4*>(dstar + (int64_t)k * E + e0));
      const float4 yv = *reinterpret_cast<const float4*>(y0 + e0);
      float4 out;
      if constexpr (kF64) {
        double a0 = promote(yv.x), a1 = promote(yv.y), a2 = promote(yv.z), a3 = promote(yv.w);
#pragma unroll
        for (int k = 0; k < GBS_MAX_SEQ; ++k)
          if (k < s.m) {
            const double c = s.c[k];
            a0 = fma(c, promote(d[k].x), a0);
            a1 = fma(c, promote(d[k].y), a1);
            a2 = fma(c, promote(d[k].z), a2);
            a3 = fma(c, promote(d[k].w), a3);
          }
        out = make_float4((float)a0, (float)a1, (float)a2, (float)a3);
      } else {
        float4 sh = yv, sl = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int k = 0; k < GBS_MAX_SEQ; ++k)
          if (k < s.m) {
            pair_combine_add(s.chi[k], s.clo[k], d[k].x, sh.x, sl.x);
            pair_combine_add(s.chi[k], s.clo[k], d[k].y, sh.y, sl.y);
            pair_combine_add(s.chi[k], s.clo[k], d[k].z, sh.z, sl.z);
            pair_combine_add(s.chi[k], s.clo[k], d[k].w, sh.w, sl.w);
          }
        out = make_float4(sh.x + sl.x, sh.y + sl.y, sh.z + sl.z, sh.w + sl.w);
      }
      *reinterpret_cast<float4*>(y_out + e0) = out;
    } else {
      for (int64_t e = e0; e <= e3; ++e) {
        const SlotDev& s = slots[probs[problem_of(probs, batch, e)].slot];
        if constexpr (kF64) {
          double a = promote(y0[e]);
          for (int k = 0; k < s.m; ++k) a = fma(s.c[k], promote(__ldcs(dstar + (int64_t)k * E + e)), a);
          y_out[e] = (float)a;
        } else {
          float sh = y0[e], sl = 0.f;
          for (int k = 0; k < s.m; ++k) pair_combine_add(s.chi[k], s.clo[k], __ldcs(dstar + (int64_t)k * E + e), sh, sl);
          y_out[e] = sh + sl;
        }
      }
    }
  }
}

// A partial step's combine share: partial = sum_k c_k d*_k over the sequences in mask (FP64,
// ascending k, the averages promoted exactly), without y_0; the sum of every rank's share is
// finished by finish_partial.
__global__ void __launch_bounds__(256) k_combine_partial(const ProbDev* probs, int batch, const SlotDev* slots,
                                                         const float* __restrict__ dstar, int64_t E, uint32_t mask,
                                                         double* __restrict__ partial) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    const SlotDev& s = slots[probs[problem_of(probs, batch, e)].slot];
    double a = 0.0;
    for (int k = 0; k < s.m; ++k)
      if ((mask >> k) & 1u) a = fma(s.c[k], promote(__ldcs(dstar + (int64_t)k * E + e)), a);
    partial[e] = a;
  }
}

size_t ring_bytes(int R, bool x2) {
  const int u = 2 * R + 1;
  if (x2) return (size_t)(kTX2 * u * kRow + u * kThreads) * sizeof(float4);
  return (size_t)(kTMax * u * kRow) * sizeof(float2);
}

// GBS_F32X2: y_out (FP64) = sum_k c_k y*_k from the averages held as FP32 pairs, summed in
// ascending k in compensated FP32 pairs as the FP32 path does (pair_combine_add on the hi parts,
// c_hi times the lo parts into the low word; error about 2^-48 of sum_k |c_k y*_k|) and rounded
// to FP64 once.  An FP64 sum spent 1.08 ms of a 9.3 ms 2048^2 macro-step on GB300's FP64 pipe.
__global__ void __launch_bounds__(256) k_combine_x2(const ProbDev* probs, int batch, const SlotDev* slots,
                                                    const float2* __restrict__ ystar, int64_t E,
                                                    double* __restrict__ y_out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    const SlotDev& s = slots[probs[problem_of(probs, batch, e)].slot];
    float sh = 0.f, sl = 0.f;
    for (int k = 0; k < s.m; ++k) {
      const float2 v = __ldcs(ystar + (int64_t)k * E + e);
      pair_combine_add(s.chi[k], s.clo[k], v.x, sh, sl);
      sl = fmaf(s.chi[k], v.y, sl);
    }
    y_out[e] = (double)sh + (double)sl;
  }
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
  float* init = nullptr;   // [2][E]: copy of y_0, f0 (written by the f0 kernel)
  float4* aux = nullptr;   // FP32: (kappa, b, f0_p, f0_u) per point (written by the f0 kernel)
  fused::Item* items = nullptr;
  int* deps = nullptr;
  int* done = nullptr;   // n_items flags followed by the queue counter
  fused::PassDesc* pdesc = nullptr;
  fused::TileGeo* tgeo = nullptr;
  size_t lev_cap = 0, ystar_cap = 0, items_cap = 0, init_cap = 0, aux_cap = 0;
  bool x2 = false;        // GBS_F32X2: levels, averages and inputs as FP32 pairs
  double alg_bytes = 0;   // algorithmic bytes of one k_passes launch
  int combine_f64 = 1;    // FP32 states: combine in FP64 (1) or in compensated FP32 pairs (0)
  uint32_t seq_mask = ~0u;   // the sequences the prepared schedule computes
  long long spin_limit = fused::kSpinLimit;
  int inject_wait = 0;    // test hook: item 0 also waits on a flag that nothing sets
};

namespace {

void free_work(FusedWork* w) {
  void* ptrs[] = {w->lev, w->ystar, w->init, w->aux, w->items, w->deps, w->done, w->pdesc, w->tgeo};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  w->lev = w->ystar = w->init = nullptr;
  w->aux = nullptr;
  w->init_cap = w->aux_cap = 0;
  w->items = nullptr;
  w->deps = w->done = nullptr;
  w->pdesc = nullptr;
  w->tgeo = nullptr;
  w->lev_cap = w->ystar_cap = w->items_cap = 0;
}

// Leap-frog levels of sequence N split into passes: first N mod tmax (if nonzero), then tmax each.
std::vector<int> pass_plan(int N, int tmax) {
  std::vector<int> v;
  int rem = N % tmax;
  if (rem) v.push_back(rem);
  for (int l = rem; l < N; l += tmax) v.push_back(tmax);
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
  if (p.system != GBS_ACOUSTIC || p.ndim != 2 || (p.f64 && !p.ds) || (p.R != 2 && p.R != 3)) return false;
  const int halo = p.R * (p.ds ? fused::kTX2 : fused::kTMax);
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

int fused_max_levels() { return fused::kTMax; }

void fused_set_combine(FusedWork* w, int f64) { w->combine_f64 = f64 != 0; }

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

int fused_prepare(FusedWork* w, const StepPlan& p, const ProbDev* probs_h, const SlotDev* slots_h,
                  const FusedTune& tune, char* msg, size_t msglen) {
  using namespace fused;
  const int hseg = tune.hseg, tmax = p.ds ? kTX2 : tune.tmax;   // pair passes: two levels
  w->x2 = p.ds != 0;
  const size_t esz = w->x2 ? 8 : 4;
  if (tmax < 2 || tmax > kTMax || tmax % 2) {
    std::snprintf(msg, msglen, "tmax must be even and in [2, %d]", kTMax);
    return -1;
  }
  w->E = p.state_elems;
  w->R = p.R;
  w->seq_mask = tune.seq_mask;
  w->hseg = hseg;
  w->m_max = p.max_m;
  // pass descriptors per (slot, seq, pass)
  std::vector<PassDesc> pdesc((size_t)GBS_MAX_SLOTS * GBS_MAX_SEQ * kMaxPasses);
  std::memset(pdesc.data(), 0, pdesc.size() * sizeof(PassDesc));
  for (int sl = 0; sl < GBS_MAX_SLOTS; ++sl)
    for (int k = 0; k < slots_h[sl].m; ++k) {
      const std::vector<int> pl = pass_plan(slots_h[sl].steps[k], tmax);
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
    tg[q] = tiles_of(probs_h[q].n[0], probs_h[q].n[1], hseg, p.R * tmax);
    const SlotDev& s = slots_h[probs_h[q].slot];
    for (int k = 0; k < s.m; ++k) {
      if (!((tune.seq_mask >> k) & 1u)) continue;   // a partial step leaves it to another rank
      const int np = (int)pass_plan(s.steps[k], tmax).size();
      for (int qq = 0; qq < np; ++qq)
        for (int t = 0; t < tg[q].nst * tg[q].nseg; ++t) keys.push_back({np - qq, q, k, qq, t});
    }
  }
  // every item's dependencies (same sequence, previous pass) come earlier in either order
  if (tune.schedule == 0)
    std::stable_sort(keys.begin(), keys.end(), [](const Key& a, const Key& b) {
      if (a.depth != b.depth) return a.depth > b.depth;
      return a.pass < b.pass;
    });
  else
    std::stable_sort(keys.begin(), keys.end(), [](const Key& a, const Key& b) {
      if (a.pass != b.pass) return a.pass < b.pass;
      return a.depth > b.depth;
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
        const int np = (int)pass_plan(s.steps[k], tmax).size();
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
  const size_t lev_bytes = (size_t)4 * p.max_m * p.state_elems * esz;
  const size_t ys_bytes = (size_t)p.max_m * p.state_elems * esz;
  const size_t init_bytes = (size_t)2 * p.state_elems * esz;
  const size_t aux_bytes =
      (size_t)(probs_h[p.batch - 1].media_off + probs_h[p.batch - 1].pts) * sizeof(float4);
  if (grow(&w->lev, &w->lev_cap, lev_bytes) || grow(&w->ystar, &w->ystar_cap, ys_bytes) ||
      grow(&w->init, &w->init_cap, init_bytes) || (!w->x2 && grow(&w->aux, &w->aux_cap, aux_bytes))) {
    std::snprintf(msg, msglen, "cudaMalloc of the fused level store (%zu bytes) failed",
                  lev_bytes + ys_bytes + init_bytes + aux_bytes);
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
  // algorithmic bytes per launch: every item reads the two media over its tile once and its two
  // input levels, and writes two levels (one average); FP32 states in increment form also read
  // f0 (a first pass reads only the media and f0: its input levels are 0 and h f0), FP32 pairs
  // read (y_0, f0) in a first pass
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
      const double rd = w->x2 ? 2.0 * p.F + 2.0 : (d.first ? 0.0 : 2.0 * p.F) + p.F + 2.0;
      by += pts * (double)esz * (rd + (d.last ? 1.0 : 2.0) * p.F);
    }
    w->alg_bytes = by;
  }
  // persistent grid: resident CTAs per SM times SMs
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = ring_bytes(p.R, w->x2);
  auto occupancy = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  };
  // The occupancy calculator answers 1 CTA per SM for any kernel that allocates tensor memory
  // (it cannot know how many columns), so for the FP32 sweep the residency is derived from its
  // registers and shared memory instead: kMinBlocks CTAs of kTmemCols columns each fit the
  // SM's 512 columns, and a tensor-memory CTA is co-resident with another once it has
  // relinquished its allocation right (k_passes does so right after allocating).
  auto residency = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncAttributes fa;
    int regs_sm = 0, smem_sm = 0, smem_res = 0;
    cudaFuncGetAttributes(&fa, kern);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_res, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    const int by_regs = regs_sm / std::max(1, ((fa.numRegs + 7) / 8) * 8 * kThreads);
    const int by_smem = smem_sm / (int)(smem + fa.sharedSizeBytes + smem_res);
    per_sm = std::min({kMinBlocks, by_regs, by_smem, 512 / kTmemCols});
  };
  if (w->x2) {
    if (p.R == 2) occupancy(k_passes<2, true>);
    else occupancy(k_passes<3, true>);
  } else {
    if (p.R == 2) residency(k_passes<2, false>);
    else residency(k_passes<3, false>);
  }
  if (cudaGetLastError() != cudaSuccess || per_sm < 1) {
    std::snprintf(msg, msglen, "the fused kernel cannot be resident (smem %zu bytes)", smem);
    return -3;
  }
  w->grid = std::max(1, std::min(n, sms * per_sm));
  return 0;
}

namespace {
// f0 (and the pair inputs) and the pass kernel of one macro-step; returns launches or -1
int fused_passes(FusedWork* w, const StepPlan& p, const void* y_in, cudaStream_t s, int* err);
}

int fused_macro_step(FusedWork* w, const StepPlan& p, const void* y_in, void* y_out, cudaStream_t s, int* err) {
  using namespace fused;
  int launches = fused_passes(w, p, y_in, s, err);
  if (launches < 0) return -1;
  if (w->x2)
    k_combine_x2<<<1024, 256, 0, s>>>(p.probs, p.batch, p.slots, reinterpret_cast<const float2*>(w->ystar), w->E,
                                      static_cast<double*>(y_out));
  else if (w->combine_f64)
    k_combine<true><<<1024, 256, 0, s>>>(p.probs, p.batch, p.slots, w->ystar, w->E, static_cast<const float*>(y_in),
                                         static_cast<float*>(y_out));
  else
    k_combine<false><<<1024, 256, 0, s>>>(p.probs, p.batch, p.slots, w->ystar, w->E, static_cast<const float*>(y_in),
                                          static_cast<float*>(y_out));
  ++launches;
  if (cudaPeekAtLastError() != cudaSuccess) return -1;
  return launches;
}

int fused_partial_step(FusedWork* w, const StepPlan& p, const void* y_in, double* partial, cudaStream_t s, int* err) {
  using namespace fused;
  if (w->x2) return -1;
  int launches = fused_passes(w, p, y_in, s, err);
  if (launches < 0) return -1;
  k_combine_partial<<<1024, 256, 0, s>>>(p.probs, p.batch, p.slots, w->ystar, w->E, w->seq_mask, partial);
  ++launches;
  if (cudaPeekAtLastError() != cudaSuccess) return -1;
  return launches;
}

namespace {
int fused_passes(FusedWork* w, const StepPlan& p, const void* y_in, cudaStream_t s, int* err) {
  using namespace fused;
  int launches = 0;
  if (w->x2) {
    // y_in, kappa and b as FP32 pairs, f0 in pair arithmetic, y_0 and f0 E pairs apart
    const int l = ds_prologue(p, y_in, w->init, reinterpret_cast<float2*>(w->init) + w->E, s);
    if (l < 0) return -1;
    launches += l;
  } else {
    // f0 goes next to a copy of y_0, and the media are interleaved for the passes
    StepPlan pf = p;
    pf.f0 = w->init + w->E;
    pf.f0_aux = w->aux;      // increment form: y_0 is read only by the combine, from y_in
    if (launch_f0(pf, y_in, s) < 0) return -1;
    ++launches;
  }
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
  P.hkq = p.hkq;
  P.aux = w->aux;
  P.init = w->init;
  P.lev = w->lev;
  P.ystar = w->ystar;
  P.E = w->E;
  P.pdesc = w->pdesc;
  P.tgeo = w->tgeo;
  P.spin_limit = w->spin_limit;
  P.kap2 = static_cast<const dsf*>(p.ds_kappa);
  P.b2 = static_cast<const dsf*>(p.ds_b);
  const size_t smem = ring_bytes(w->R, w->x2);
  const int u = timing_begin(p, s);
  if (w->x2) {
    if (w->R == 2) k_passes<2, true><<<w->grid, kThreads, smem, s>>>(P);
    else k_passes<3, true><<<w->grid, kThreads, smem, s>>>(P);
  } else {
    if (w->R == 2) k_passes<2, false><<<w->grid, kThreads, smem, s>>>(P);
    else k_passes<3, false><<<w->grid, kThreads, smem, s>>>(P);
  }
  timing_end(p, u, s, w->alg_bytes);
  ++launches;
  if (cudaPeekAtLastError() != cudaSuccess) return -1;
  return launches;
}
}  // namespace

}  // namespace gbs
