// Internal declarations shared by the host library and its CUDA kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gbs.h"

namespace gbs {

constexpr int kMaxFields = 4;

// One problem of a batch, as the kernels see it.
struct ProbDev {
  int n[3];            // nx, ny, nz (unused dims = 1)
  int slot;            // weight slot
  int64_t pts;         // nx * ny * nz
  int64_t state_off;   // element offset of the problem's [F][nz][ny][nx] block
  int64_t media_off;   // element offset of its [nz][ny][nx] media block
  int64_t blk_begin;   // first block of this problem in a point-parallel grid
  int64_t tblk_begin;  // first block of this problem in the x-y tiled grid
  int tiles_x, tiles_y;  // x-y tiles per z plane (kTileX x kTileY points each)
  double inv_dx[3];
  // FP32 kernels (integer-weight stencil sums, gbs_plain.cu): dx_0 / dx_d per axis, and
  // 1 / (div dx_0) split into two floats (div = 12 or 60, the weights' common divisor)
  float rr[3];
  float f0s[2];
};

// The FP32 kernels' per-problem constants above (host; R the stencil radius).
inline void fill_fp32_consts(ProbDev& q, int ndim, int R) {
  for (int d = 0; d < 3; ++d) q.rr[d] = d < ndim ? (float)(q.inv_dx[d] / q.inv_dx[0]) : 0.f;
  const double c = q.inv_dx[0] / (R == 2 ? 12.0 : 60.0);
  q.f0s[0] = (float)c;
  q.f0s[1] = (float)(c - (double)q.f0s[0]);
}

// The FP32 kernels' per-sequence step constants (host): 2h and 2h / (div dx_0) of sequence k of
// problem q, each split into two floats (hi, lo).
inline float4 fp32_step_consts(const ProbDev& q, double hk, int R) {
  const double g = 2.0 * hk, sc = g * q.inv_dx[0] / (R == 2 ? 12.0 : 60.0);
  const float gh = (float)g, sh = (float)sc;
  return make_float4(gh, (float)(g - (double)gh), sh, (float)(sc - (double)sh));
}

// One weight slot: m sequences with step counts and FP64 weights, in
// combine order (dependent weights first, then free ones).
struct SlotDev {
  int m;
  int steps[GBS_MAX_SEQ];
  double c[GBS_MAX_SEQ];
  float chi[GBS_MAX_SEQ];   // c = chi + clo (+ O(2^-48 c)): the weights split for FP32-pair sums
  float clo[GBS_MAX_SEQ];
};

// Fill chi/clo from c (host).
inline void split_weights(SlotDev& s) {
  for (int k = 0; k < GBS_MAX_SEQ; ++k) {
    s.chi[k] = (float)s.c[k];
    s.clo[k] = (float)(s.c[k] - (double)s.chi[k]);
  }
}

// Everything a macro-step launcher needs (device pointers except where noted).
struct StepPlan {
  int system, ndim, R, f64;    // f64: 1 = FP64 states and media in the API (GBS_F64, GBS_F32X2)
  int ds;                      // 1 = GBS_F32X2: levels and right-hand sides in FP32 pairs
  int F;
  int batch;
  const ProbDev* probs;
  const SlotDev* slots;
  const double* H;             // per problem
  const double* hk;            // per problem x GBS_MAX_SEQ: h_k = H / N_k (host-computed)
  const float2* hkf;           // the same as FP32 pairs (h_k, 2 h_k)
  const float4* hkq;           // FP32 paths, per problem x GBS_MAX_SEQ: fp32_step_consts
  int64_t total_blocks;        // point-parallel blocks over the whole batch
  int64_t total_tiles;         // x-y tiled blocks over the whole batch (2D/3D)
  int64_t state_elems;         // scalars in one state buffer (sum of F * pts)
  int64_t probs_media_elems;   // scalars in one media array (sum of pts)
  int64_t max_nx;              // largest nx over the problems
  int nx_vec;                  // 1 = every problem's nx is a multiple of 4, so every row of every
                               // state buffer starts on a 16-byte boundary (vector staging)
  const void* kappa;           // media (state element type)
  const void* b;               // 1 / rho
  void* f0;                    // shared first RHS, F x P
  void* L0;                    // leap-frog level buffers, F x P each
  void* L1;
  double* acc;                 // FP64 combine accumulator, F x P
  // optional output of the f0 kernel (FP32 2D acoustics, time-blocked path): per point
  // (kappa, b, f0_p, f0_u) interleaved, f0_v in the f0 buffer's third field (its first two
  // fields are then not written)
  float4* f0_aux;
  // GBS_F32X2 workspace: y_in, kappa and b converted to FP32 pairs at the start of a step
  void* ds_y0;
  void* ds_kappa;
  void* ds_b;
  // host-side schedule: for sequence index k, the largest step count over problems
  int max_m;
  int max_steps_k[GBS_MAX_SEQ];
  // optional kernel timing (host pointers): event pairs around each dominant-kernel
  // launch, and the algorithmic bytes of that launch
  cudaEvent_t* tev;
  double* tev_bytes;
  int tev_cap;
  int* tev_used;
  const int64_t* active_pts;   // [k * (GBS_MAX_STEPS + 1) + n]: points updated by step (k, n)
  double unit_bytes;           // algorithmic bytes per grid-point update of the dominant kernel
  double adj_unit_bytes;       // the same for the adjoint's reverse step (k_adj_rev)
  // tensor-map (TMA) staging of the FP32 tiled leap-frog step: host pointers to the 128-byte
  // maps of the level buffers L0 and L1 (NULL: stage with loads), and the device error flag a
  // bounded wait on the copy latches GBS_ERR_TIMEOUT in
  const void* lf_tmap[2];
  int* err;
  // sequence-parallel partial steps: bit k set = sequence k of every problem's slot is computed
  // (all bits: a whole macro-step); partial = 1: the combine accumulates only those sequences'
  // share in acc (no y_0 term, no y_out written)
  uint32_t seq_mask;
  int partial;
};

// First and last sequence a step computes among the slot's m sequences (device).
__device__ __forceinline__ void seq_first_last(const StepPlan& p, int k, int m, bool& first, bool& last) {
  const unsigned msk = p.seq_mask & ((1u << m) - 1u);   // m <= GBS_MAX_SEQ = 16
  first = k == __ffs(msk) - 1;
  last = !p.partial && k == 31 - __clz(msk);
}

// Tensor map of one FP32 level buffer [F][nz][ny][nx] for the tiled leap-frog step's staging
// box (the tile's 40 staged columns x 32 + 2R rows x one z-plane x the fields p, u, v); writes
// the 128-byte map to `map`.  Requires nx % 4 == 0 and a 16-byte aligned base.  Returns 0, or
// -1 when the driver entry point or the encoding is unavailable (the kernel then stages with
// loads).
int lf_tma_encode(void* map, void* base, int nx, int ny, int nz, int F, int R);

// Record the start of a timed launch; returns the slot index or -1.
inline int timing_begin(const StepPlan& p, cudaStream_t s) {
  if (!p.tev || *p.tev_used >= p.tev_cap) return -1;
  const int u = (*p.tev_used)++;
  cudaEventRecord(p.tev[2 * u], s);
  return u;
}
inline void timing_end(const StepPlan& p, int u, cudaStream_t s, double bytes) {
  if (u < 0) return;
  cudaEventRecord(p.tev[2 * u + 1], s);
  p.tev_bytes[u] = bytes;
}

constexpr int kPlainBlock = 256;
constexpr int kSpectralMaxN = 2048;   // GBS_ONEWAY_SPECTRAL: one problem's macro-step per block

// One-way wave with spectral derivatives (gbs_spectral.cu): one macro-step of every problem,
// one block per problem; returns the number of kernels launched or -1.
int spectral_macro_step(const StepPlan& p, const void* y_in, void* y_out, cudaStream_t s);
int spectral_setup();   // opt the kernel into its shared memory (handle creation, not in a capture)
constexpr int kTileX = 32;   // tiled step kernels: 32 x 8 threads, 4 rows per thread
constexpr int kTileRows = 4;
constexpr int kTileY = 8 * kTileRows;

// Fill the tiled-grid fields of a problem table (host); returns the total tile count.
inline int64_t assign_tiles(ProbDev* probs, int batch, int ndim) {
  int64_t t = 0;
  for (int i = 0; i < batch; ++i) {
    ProbDev& q = probs[i];
    q.tiles_x = (q.n[0] + kTileX - 1) / kTileX;
    q.tiles_y = ndim >= 2 ? (q.n[1] + kTileY - 1) / kTileY : 1;
    q.tblk_begin = t;
    t += (int64_t)q.tiles_x * q.tiles_y * q.n[2];
  }
  return t;
}

// Enqueue one plain macro-step (y_in -> y_out) on `s`.  Returns the number of
// kernels launched, or -1 if a launch failed (cudaGetLastError set).
int plain_macro_step(const StepPlan& p, const void* y_in, void* y_out, cudaStream_t s);

// f0 = f(y_in) for every problem (point-parallel); returns 1 or -1.
int launch_f0(const StepPlan& p, const void* y_in, cudaStream_t s);

// GBS_F32X2 inputs of the time-blocked path: y_in (FP64) as FP32 pairs at y_pairs, kappa and b as
// pairs at p.ds_kappa / p.ds_b, and f0 = f(y_in) in pair arithmetic at f0_pairs (acoustics).
// Returns the number of kernels launched, or -1.
int ds_prologue(const StepPlan& p, const void* y_in, void* y_pairs, void* f0_pairs, cudaStream_t s);

// Time-blocked path for 2D acoustics (gbs_fused.cu): FP32 states, or FP64 states in FP32 pairs
// (GBS_F32X2).  FusedWork holds its
// schedule and level store; fused_prepare (set-up time) allocates them.
struct FusedWork;
FusedWork* fused_create();
// spin_limit: polls before a dependency wait gives up (GBS_ERR_TIMEOUT); inject_wait: test
// hook making the first item wait on a flag that nothing sets (takes effect at prepare).
void fused_set_test_hooks(FusedWork* w, long long spin_limit, int inject_wait);
// FP32 states: sum the combine in FP64 (f64 = 1, the default) or in compensated FP32 pairs (0).
void fused_set_combine(FusedWork* w, int f64);
void fused_destroy(FusedWork* w);
bool fused_supported(const StepPlan& p, const ProbDev* probs_h);
// Tunable shape of the time-blocked schedule: row-segment height of a tile, the most leap-frog
// levels per pass (even, 2..4), and the queue order (0: longest remaining chain of passes
// first; 1: pass by pass, all sequences' first passes first).
struct FusedTune {
  int hseg;
  int tmax;
  int schedule;
  uint32_t seq_mask;   // sequences scheduled (bit k: sequence k); all bits for whole macro-steps
};
int fused_prepare(FusedWork* w, const StepPlan& p, const ProbDev* probs_h, const SlotDev* slots_h,
                  const FusedTune& tune, char* msg, size_t msglen);
int fused_max_levels();   // largest tmax the kernel was compiled for
int fused_macro_step(FusedWork* w, const StepPlan& p, const void* y_in, void* y_out, cudaStream_t s, int* err);
// FP32 states: the sequences of the prepared mask only, their combine share written to partial
// (FP64, state layout): sum_k c_k d*_k over those sequences.
int fused_partial_step(FusedWork* w, const StepPlan& p, const void* y_in, double* partial, cudaStream_t s, int* err);
// y_out = y_in (increment form) or 0 (others) + total, total the FP64 sum of every rank's partial
int finish_partial(const StepPlan& p, const void* y_in, const double* total, void* y_out, cudaStream_t s);

// Adjoint of one macro-step with stored forward levels (plain kernels).
struct AdjPlan {
  StepPlan fw;
  void* levels;                // (max_steps + 2) x F x P forward levels
  void* mu0;                   // two adjoint level buffers, F x P each
  void* mu1;
  void* shared;                // sum_k h_k mu_1^k, F x P (state type)
  float2* gpair;               // FP32 path: the macro-step's reverse-step gradient terms, (hi, lo) per point
  int max_steps;
  int64_t rcv_pts;             // valid receiver indices: [0, rcv_pts)
  int* err;                    // device error flag
};
int plain_adjoint_step(const AdjPlan& p, const void* y_in, const void* lam_out, void* lam_in,
                       double* grad_kappa, const int64_t* rcv_idx, int n_rcv,
                       const void* rcv_resid, cudaStream_t s);

// Media preparation and reductions (gbs_reduce.cu).
int prep_media(int f64, const void* rho, void* b, int64_t n, cudaStream_t s);
// max over each problem of sqrt(kappa * b): out[batch] (device double), scratch >= batch*1024 doubles
int media_cmax(int f64, const void* kappa, const void* b, const ProbDev* probs, int batch,
               double* out, cudaStream_t s);
// norms: out4 device doubles; partial: device scratch of >= 4 * kNormBlocks doubles
constexpr int kNormBlocks = 1024;
int norms(int f64, const void* a, const void* b, int64_t n, double* partial, double* out4,
          cudaStream_t s);
int inject(int f64, void* lam, const int64_t* idx, int n, const void* values, int64_t n_valid, int* err,
           cudaStream_t s);
int misfit(int f64, const void* y, const int64_t* idx, int n_rcv, const void* data, void* resid,
           double* J, int64_t n_valid, int* err, cudaStream_t s);

}  // namespace gbs
