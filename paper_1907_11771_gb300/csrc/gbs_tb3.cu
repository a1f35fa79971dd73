// Time-blocked leap-frog passes for 3D acoustics with FP32 states (increment form).
//
// The leap-frog levels of sequence k (Sec. 2.1 eq. "GBS": y_(n+1) = y_(n-1) + 2 h f(y_n),
// n = 1 .. N_k, after the Forward-Euler level y_1) are advanced two per pass: pass j reads the
// levels (d_(2j), d_(2j+1)) of the whole grid and writes (d_(2j+2), d_(2j+3)), or, in the
// sequence's last pass, adds c_k times Gragg's average (d_(N-1) + 2 d_N + d_(N+1)) / 4 to the
// FP64 combine (Sec. 3.2).  Pass 0 starts from d_0 = 0 and d_1 = h f0 (f0 = f(y_0), shared by
// every sequence, Sec. 3.6), so no level of the Forward-Euler step is stored.  One pass reads
// two levels, f0 and the media and writes two levels: 22 floats per point for two updates, where
// the one-level kernel moves 18 floats per update.  Passes alternate between two buffer pairs,
// so a pass never overwrites what another block of it still reads.
//
// Inside a pass (one block per x-y tile and z-segment, one grid column (x, y) per thread) the
// block sweeps its segment plane by plane with a time skew: at sweep step s, level 0 (the
// pass's input d_(2j+1)) enters plane zL = z_a - 2R + s, level 1 (d_(2j+2)) computes plane
// zL - R and level 2 (d_(2j+3)) plane zL - 2R, each R planes behind the level it reads, the
// reach of the z-stencils.  Every thread keeps its column's last 2R + 1 planes of level 0 (all
// fields: the z-stencils of p and w, and level 2's leap-frog "previous" value) and of level 1
// (p and w; u and v for R + 1 planes) in registers.  The x- and y-stencils read the neighbours'
// values from two shared planes per step (level 0 at zL - R, level 1 at zL - 2R), double
// buffered so that one barrier per step suffices.  Level 1 is valid on the tile shrunk by R on
// every side and level 2 on the tile shrunk by 2R, which is what the block writes.
//
// The arithmetic of every update is that of the one-level kernel (integer-weight stencil sums,
// pair-scaled media, the forcing 2h f0 as a split product), in the same order, so both kernels
// give the same bits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <vector>

#include "gbs_ds.cuh"
#include "gbs_internal.h"
#include "gbs_stencil.cuh"
#include "gbs_tb3.h"

namespace gbs {

struct Tb3Geo {
  int64_t begin;   // first block of the problem
  int tiles_x, tiles_y, zsegs, zlen;
};

struct Tb3Work {
  void* L2 = nullptr;   // the second level-buffer pair, state layout
  void* L3 = nullptr;
  size_t lev_elems = 0;
  Tb3Geo* d_geo = nullptr;
  int geo_cap = 0;
  int64_t total_blocks = 0;
  // per sequence k and pass j: points of the problems that run the pass
  std::vector<int64_t> pass_pts;
  int max_pass = 0;
};

namespace tb3 {

constexpr int kX = 32;            // tile columns (one warp per tile row)
constexpr int kY = 24;            // tile rows
constexpr int kThreads = kX * kY;

template <int R>
constexpr int interior_x() { return kX - 4 * R; }
template <int R>
constexpr int interior_y() { return kY - 4 * R; }

__device__ __forceinline__ int wrap_full(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

template <int R>
__global__ void __launch_bounds__(kThreads, 1)
    k_tb3(const StepPlan p, const Tb3Geo* __restrict__ geo, const float* y_in, float* y_out,
          const float* __restrict__ in0, const float* __restrict__ in1, float* __restrict__ out0,
          float* __restrict__ out1, int k, int j) {
  constexpr int W = 2 * R + 1;
  constexpr int IX = interior_x<R>(), IY = interior_y<R>();
  // [step parity][level 0 / level 1][p, u, v][row][column]
  __shared__ float S[2][2][3][kY][kX];
  int lo = 0, hi = p.batch - 1;
  const int64_t blk = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (geo[mid].begin <= blk) lo = mid;
    else hi = mid - 1;
  }
  const ProbDev& q = p.probs[lo];
  const Tb3Geo g = geo[lo];
  const SlotDev& sl = p.slots[q.slot];
  if (k >= sl.m) return;
  const int N = sl.steps[k];
  if (2 * j + 2 > N) return;   // this problem's sequence has fewer passes
  const bool pass0 = j == 0, lastp = 2 * j + 2 == N;
  int t = (int)(blk - g.begin);
  const int tx = t % g.tiles_x;
  t /= g.tiles_x;
  const int ty = t % g.tiles_y;
  const int zs = t / g.tiles_y;
  const int nx = q.n[0], ny = q.n[1], nz = q.n[2], nxy = nx * ny;
  const int lx = threadIdx.x, ly = threadIdx.y;
  const int ox = tx * IX - 2 * R + lx, oy = ty * IY - 2 * R + ly;   // the column, unwrapped
  const int col = wrap_full(oy, ny) * nx + wrap_full(ox, nx);
  const bool act1 = ly >= R && ly < kY - R && lx >= R && lx < kX - R;
  const bool act2 = ly >= 2 * R && ly < kY - 2 * R && lx >= 2 * R && lx < kX - 2 * R;
  const bool outp = act2 && ox < nx && oy < ny;
  const int za = zs * g.zlen, zb = min(nz, za + g.zlen);
  const int nsteps = (zb - za) + 4 * R;
  const int64_t P = q.pts;
  const float* f0v = static_cast<const float*>(p.f0) + q.state_off;
  const float* kap = static_cast<const float*>(p.kappa) + q.media_off;
  const float* bme = static_cast<const float*>(p.b) + q.media_off;
  const float* a0 = in0 + q.state_off;   // d_(2j)   (pass 0: zero, not read)
  const float* a1 = in1 + q.state_off;   // d_(2j+1) (pass 0: h f0, from f0)
  float* b0 = out0 + q.state_off;
  float* b1 = out1 + q.state_off;
  // the forcing's 2h and -2h / (div dx_0) as float pairs; idy, idz = dx_0 / dx_d
  const float4 hq = p.hkq[lo * GBS_MAX_SEQ + k];
  const float gh = hq.x, gl = hq.y, sch = -hq.z, scl = -hq.w;
  const float idy = q.rr[1], idz = q.rr[2];
  const double c = sl.c[k];
  bool first, last;
  seq_first_last(p, k, sl.m, first, last);

  // level 0 at planes zL - 2R .. zL (index W - 1 newest); level 1's p, w at zL - 3R .. zL - R
  // and u, v at zL - 2R .. zL - R once this step's plane is in
  float P0[W], U0[W], V0[W], W0[W], P1[W], W1[W], U1[R + 1], V1[R + 1];
#pragma unroll
  for (int i = 0; i < W; ++i) P0[i] = U0[i] = V0[i] = W0[i] = P1[i] = W1[i] = 0.f;
#pragma unroll
  for (int i = 0; i <= R; ++i) U1[i] = V1[i] = 0.f;

  auto load0 = [&](int zw, float* o) {
    const int e = zw * nxy + col;
#pragma unroll
    for (int fl = 0; fl < 4; ++fl) {
      if (pass0) o[fl] = 0.5f * mul_split(gh, gl, ldg(f0v + fl * P + e));   // d_1 = (2h f0) / 2
      else o[fl] = ldg(a1 + fl * P + e);
    }
  };
  // planes of the three levels at the current step, wrapped (periodic in z)
  int z0 = wrap_full(za - 2 * R, nz), z1 = wrap_full(za - 3 * R, nz), z2 = wrap_full(za - 4 * R, nz);
  float n0[4];
  load0(z0, n0);
  for (int s = 0; s < nsteps; ++s) {
#pragma unroll
    for (int i = 0; i + 1 < W; ++i) {
      P0[i] = P0[i + 1];
      U0[i] = U0[i + 1];
      V0[i] = V0[i + 1];
      W0[i] = W0[i + 1];
    }
    P0[W - 1] = n0[0];
    U0[W - 1] = n0[1];
    V0[W - 1] = n0[2];
    W0[W - 1] = n0[3];
    // point-wise operands of this step's two updates, issued before the barrier
    const bool do1 = s >= 2 * R, do2 = s >= 4 * R;
    const int e1 = z1 * nxy + col, e2 = z2 * nxy + col;
    float pv1[4], fa1[4], fa2[4], k1 = 0.f, m1 = 0.f, k2 = 0.f, m2 = 0.f;
#pragma unroll
    for (int fl = 0; fl < 4; ++fl) pv1[fl] = fa1[fl] = fa2[fl] = 0.f;
    if (do1 && act1) {
#pragma unroll
      for (int fl = 0; fl < 4; ++fl) {
        if (!pass0) pv1[fl] = ldg(a0 + fl * P + e1);
        fa1[fl] = ldg(f0v + fl * P + e1);
      }
      k1 = ldg(kap + e1);
      m1 = ldg(bme + e1);
    }
    if (do2 && act2) {
#pragma unroll
      for (int fl = 0; fl < 4; ++fl) fa2[fl] = ldg(f0v + fl * P + e2);
      k2 = ldg(kap + e2);
      m2 = ldg(bme + e2);
    }
    // the next step's level-0 plane
    z0 = z0 + 1 == nz ? 0 : z0 + 1;
    if (s + 1 < nsteps) load0(z0, n0);
    // publish level 0 at zL - R and level 1 at zL - 2R (computed R steps ago)
    const int buf = s & 1;
    S[buf][0][0][ly][lx] = P0[R];
    S[buf][0][1][ly][lx] = U0[R];
    S[buf][0][2][ly][lx] = V0[R];
    S[buf][1][0][ly][lx] = P1[R + 1];
    S[buf][1][1][ly][lx] = U1[1];
    S[buf][1][2][ly][lx] = V1[1];
    __syncthreads();
    if (do1) {
      // level 1 at plane zL - R
      float nv[4] = {0.f, 0.f, 0.f, 0.f};
      if (act1) {
        float sxu = 0.f, sxp = 0.f, syv = 0.f, syp = 0.f, szp = 0.f, szw = 0.f;
#pragma unroll
        for (int jj = 1; jj <= R; ++jj) {
          const float a = fd_int<R>(jj);
          sxp += a * (S[buf][0][0][ly][lx + jj] - S[buf][0][0][ly][lx - jj]);
          sxu += a * (S[buf][0][1][ly][lx + jj] - S[buf][0][1][ly][lx - jj]);
          syp += a * (S[buf][0][0][ly + jj][lx] - S[buf][0][0][ly - jj][lx]);
          syv += a * (S[buf][0][2][ly + jj][lx] - S[buf][0][2][ly - jj][lx]);
        }
#pragma unroll
        for (int jj = 1; jj <= R; ++jj) {
          const float a = fd_int<R>(jj);
          szp += a * (P0[R + jj] - P0[R - jj]);
          szw += a * (W0[R + jj] - W0[R - jj]);
        }
        float f[4];
        float sd = fmaf(idy, syv, sxu);
        sd = fmaf(idz, szw, sd);
        f[0] = sd;
        f[1] = sxp;
        f[2] = idy * syp;
        f[3] = idz * szp;
        const float kh = __fmul_rn(sch, k1);
        const float kl = fmaf(scl, k1, fmaf(sch, k1, -kh));
        const float bh = __fmul_rn(sch, m1);
        const float bl = fmaf(scl, m1, fmaf(sch, m1, -bh));
#pragma unroll
        for (int fl = 0; fl < 4; ++fl) {
          const float pg = pv1[fl] + mul_split(gh, gl, fa1[fl]);
          const float mh = fl == 0 ? kh : bh, ml = fl == 0 ? kl : bl;
          nv[fl] = fmaf(mh, f[fl], fmaf(ml, f[fl], pg));
        }
      }
#pragma unroll
      for (int i = 0; i + 1 < W; ++i) {
        P1[i] = P1[i + 1];
        W1[i] = W1[i + 1];
      }
#pragma unroll
      for (int i = 0; i < R; ++i) {
        U1[i] = U1[i + 1];
        V1[i] = V1[i + 1];
      }
      P1[W - 1] = nv[0];
      U1[R] = nv[1];
      V1[R] = nv[2];
      W1[W - 1] = nv[3];
      if (do2 && act2) {
        // level 2 at plane zL - 2R: in-plane neighbours from level 1's shared plane, z from its
        // window (centre R), the leap-frog "previous" value from level 0's oldest plane
        float sxu = 0.f, sxp = 0.f, syv = 0.f, syp = 0.f, szp = 0.f, szw = 0.f;
#pragma unroll
        for (int jj = 1; jj <= R; ++jj) {
          const float a = fd_int<R>(jj);
          sxp += a * (S[buf][1][0][ly][lx + jj] - S[buf][1][0][ly][lx - jj]);
          sxu += a * (S[buf][1][1][ly][lx + jj] - S[buf][1][1][ly][lx - jj]);
          syp += a * (S[buf][1][0][ly + jj][lx] - S[buf][1][0][ly - jj][lx]);
          syv += a * (S[buf][1][2][ly + jj][lx] - S[buf][1][2][ly - jj][lx]);
        }
#pragma unroll
        for (int jj = 1; jj <= R; ++jj) {
          const float a = fd_int<R>(jj);
          szp += a * (P1[R + jj] - P1[R - jj]);
          szw += a * (W1[R + jj] - W1[R - jj]);
        }
        float f[4];
        float sd = fmaf(idy, syv, sxu);
        sd = fmaf(idz, szw, sd);
        f[0] = sd;
        f[1] = sxp;
        f[2] = idy * syp;
        f[3] = idz * szp;
        const float kh = __fmul_rn(sch, k2);
        const float kl = fmaf(scl, k2, fmaf(sch, k2, -kh));
        const float bh = __fmul_rn(sch, m2);
        const float bl = fmaf(scl, m2, fmaf(sch, m2, -bh));
        const float pv2[4] = {P0[0], U0[0], V0[0], W0[0]};
        const float l1[4] = {P1[R], U1[0], V1[0], W1[R]};
        if (outp) {
#pragma unroll
          for (int fl = 0; fl < 4; ++fl) {
            const float pg = pv2[fl] + mul_split(gh, gl, fa2[fl]);
            const float mh = fl == 0 ? kh : bh, ml = fl == 0 ? kl : bl;
            const float d2 = fmaf(mh, f[fl], fmaf(ml, f[fl], pg));
            const int64_t e = fl * P + e2;
            if (!lastp) {
              b0[e] = l1[fl];
              b1[e] = d2;
            } else {
              combine_last<float, float, true>(p.acc + q.state_off, e, first, last, c, gragg_avg(pv2[fl], l1[fl], d2),
                           y_out + q.state_off, first && !p.partial ? y_in[q.state_off + e] : 0.f);
            }
          }
        }
      }
    }
    z1 = z1 + 1 == nz ? 0 : z1 + 1;
    z2 = z2 + 1 == nz ? 0 : z2 + 1;
  }
}

}  // namespace tb3

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

Tb3Work* tb3_create() { return new Tb3Work(); }

void tb3_destroy(Tb3Work* w) {
  if (!w) return;
  if (w->L2) cudaFree(w->L2);
  if (w->L3) cudaFree(w->L3);
  if (w->d_geo) cudaFree(w->d_geo);
  delete w;
}

size_t tb3_workspace_bytes(int64_t state_elems) { return 2 * sizeof(float) * (size_t)state_elems; }

bool tb3_supported(const StepPlan& p, const ProbDev* probs_h, const SlotDev* slots_h, int n_slots) {
  if (p.system != GBS_ACOUSTIC || p.ndim != 3 || p.f64 || p.ds || (p.R != 2 && p.R != 3)) return false;
  for (int i = 0; i < p.batch; ++i) {
    const int sl = probs_h[i].slot;
    if (sl < 0 || sl >= n_slots) return false;
    for (int k = 0; k < slots_h[sl].m; ++k)
      if (slots_h[sl].steps[k] % 2) return false;
  }
  return true;
}

int tb3_prepare(Tb3Work* w, const StepPlan& p, const ProbDev* probs_h, const SlotDev* slots_h, int zseg,
                char* msg, size_t msglen) {
  const int IX = tb3::kX - 4 * p.R, IY = tb3::kY - 4 * p.R;
  std::vector<Tb3Geo> geo(p.batch);
  int64_t t = 0;
  for (int i = 0; i < p.batch; ++i) {
    const ProbDev& q = probs_h[i];
    Tb3Geo& g = geo[i];
    g.begin = t;
    g.tiles_x = (q.n[0] + IX - 1) / IX;
    g.tiles_y = (q.n[1] + IY - 1) / IY;
    g.zlen = std::max(1, std::min(zseg, q.n[2]));
    g.zsegs = (q.n[2] + g.zlen - 1) / g.zlen;
    t += (int64_t)g.tiles_x * g.tiles_y * g.zsegs;
  }
  if (t >= (1ll << 31)) {
    snprintf(msg, msglen, "the 3D time-blocked grid has too many blocks");
    return -1;
  }
  if (w->lev_elems != (size_t)p.state_elems) {
    if (w->L2) cudaFree(w->L2);
    if (w->L3) cudaFree(w->L3);
    w->L2 = w->L3 = nullptr;
    w->lev_elems = 0;
    if (cudaMalloc(&w->L2, sizeof(float) * p.state_elems) != cudaSuccess ||
        cudaMalloc(&w->L3, sizeof(float) * p.state_elems) != cudaSuccess) {
      cudaGetLastError();
      snprintf(msg, msglen, "cudaMalloc of the 3D time-blocked level buffers (%lld bytes) failed",
               (long long)(2 * sizeof(float) * p.state_elems));
      return -2;
    }
    w->lev_elems = (size_t)p.state_elems;
  }
  if (w->geo_cap < p.batch) {
    if (w->d_geo) cudaFree(w->d_geo);
    w->d_geo = nullptr;
    w->geo_cap = 0;
    if (cudaMalloc(&w->d_geo, sizeof(Tb3Geo) * p.batch) != cudaSuccess) {
      cudaGetLastError();
      snprintf(msg, msglen, "cudaMalloc of the 3D tile table failed");
      return -2;
    }
    w->geo_cap = p.batch;
  }
  if (cudaMemcpy(w->d_geo, geo.data(), sizeof(Tb3Geo) * p.batch, cudaMemcpyHostToDevice) != cudaSuccess) {
    snprintf(msg, msglen, "upload of the 3D tile table failed");
    return -1;
  }
  w->total_blocks = t;
  w->max_pass = GBS_MAX_STEPS / 2;
  w->pass_pts.assign((size_t)GBS_MAX_SEQ * w->max_pass, 0);
  for (int i = 0; i < p.batch; ++i) {
    const SlotDev& s = slots_h[probs_h[i].slot];
    for (int k = 0; k < s.m; ++k)
      for (int j = 0; 2 * j + 2 <= s.steps[k]; ++j) w->pass_pts[(size_t)k * w->max_pass + j] += probs_h[i].pts;
  }
  return 0;
}

namespace {

// algorithmic bytes of one point of pass j: reads d_(2j) and d_(2j+1) (pass 0: neither), f0 and
// the media; writes two levels, or in the last pass the FP64 combine (accumulator read unless
// first, written unless last, then y_out; the first sequence reads y_0)
double pass_bytes(int F, bool pass0, bool lastp) {
  double b = 4.0 * ((pass0 ? 0 : 2 * F) + F + 2);
  b += lastp ? 0.5 * (8.0 * F + 8.0 * F) : 8.0 * F;
  return b;
}

}  // namespace

int tb3_macro_step(const Tb3Work* w, const StepPlan& p, const void* y_in_v, void* y_out_v, cudaStream_t st) {
  if (!w || !w->d_geo || !w->L2 || w->total_blocks <= 0) return -1;
  const float* y_in = static_cast<const float*>(y_in_v);
  float* y_out = static_cast<float*>(y_out_v);
  if (launch_f0(p, y_in_v, st) < 0) return -1;
  int launches = 1;
  const dim3 block(tb3::kX, tb3::kY);
  float* set[2][2] = {{static_cast<float*>(p.L0), static_cast<float*>(p.L1)},
                      {static_cast<float*>(w->L2), static_cast<float*>(w->L3)}};
  for (int k = 0; k < p.max_m; ++k) {
    if (!((p.seq_mask >> k) & 1u)) continue;
    const int npass = p.max_steps_k[k] / 2;
    for (int j = 0; j < npass; ++j) {
      float* const* in = set[j & 1];
      float* const* out = set[(j + 1) & 1];
      const int u = timing_begin(p, st);
      if (p.R == 2)
        tb3::k_tb3<2><<<(unsigned)w->total_blocks, block, 0, st>>>(p, w->d_geo, y_in, y_out, in[0], in[1], out[0],
                                                                   out[1], k, j);
      else
        tb3::k_tb3<3><<<(unsigned)w->total_blocks, block, 0, st>>>(p, w->d_geo, y_in, y_out, in[0], in[1], out[0],
                                                                   out[1], k, j);
      if (u >= 0) {
        // points of this pass: the problems whose sequence k runs it (the last pass of some,
        // a middle pass of others is counted at the middle-pass rate)
        const int64_t pts = w->pass_pts[(size_t)k * w->max_pass + j];
        const bool lastp = 2 * j + 2 == p.max_steps_k[k];
        timing_end(p, u, st, (double)pts * pass_bytes(p.F, j == 0, lastp));
      }
      ++launches;
    }
  }
  if (cudaPeekAtLastError() != cudaSuccess) return -1;
  return launches;
}

}  // namespace gbs
