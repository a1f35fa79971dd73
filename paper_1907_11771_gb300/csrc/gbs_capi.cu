// C ABI of the GBS library: handle life cycle, validation, scheme set-up
// (weights, order constraints, stability boundary), workspace, and the
// dispatch of macro-steps (with CUDA-graph replay) and adjoint steps.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "gbs_dd.h"
#include "gbs_internal.h"
#include "gbs_seqfuse.h"
#include "gbs_tb3.h"
#include "gbs_weights.h"

using namespace gbs;

namespace {

thread_local std::string g_create_error;

struct Slot {
  bool set = false;
  int order = 0;
  int m = 0;
  int steps[GBS_MAX_SEQ] = {0};
  double c[GBS_MAX_SEQ] = {0};
  double isb = 0;
};

struct GraphEntry {
  const void* yi = nullptr;
  void* yo = nullptr;
  int kernel = 0;
  uint64_t version = 0;
  cudaGraphExec_t exec = nullptr;
  int launches = 0;
};

}  // namespace

struct gbs_ctx {
  // problem
  int system = 0, ndim = 0, order = 0, R = 0, f64 = 0, batch = 0, F = 0, adjoint = 0;
  int ds = 0;                             // GBS_F32X2: FP32-pair levels and right-hand sides
  size_t esz = 4;                         // state element size
  std::vector<ProbDev> probs;
  int64_t state_elems = 0, media_elems = 0, total_blocks = 0, total_tiles = 0;
  std::vector<double> cmax;               // per problem max sqrt(kappa b)
  // media
  const void* kappa = nullptr;
  void* b = nullptr;
  // slots
  Slot slots[GBS_MAX_SLOTS];
  std::vector<int> slot_of;
  // device tables
  ProbDev* d_probs = nullptr;
  SlotDev* d_slots = nullptr;
  double* d_H = nullptr;
  double* d_hk = nullptr;                 // per problem x GBS_MAX_SEQ: H / N_k
  float2* d_hkf = nullptr;                // the same as FP32 (h_k, 2 h_k)
  float4* d_hkq = nullptr;                // FP32 kernels' split step constants (fp32_step_consts)
  std::vector<double> cur_H;
  std::vector<double> hk_host;
  std::vector<float2> hkf_host;
  std::vector<float4> hkq_host;
  int* d_err = nullptr;
  double* d_red = nullptr;                // norm partials (4 * kNormBlocks) + 4 results
  double* d_cmax = nullptr;
  // workspace
  void* f0 = nullptr;
  void* L0 = nullptr;
  void* L1 = nullptr;
  double* acc = nullptr;
  void* stage = nullptr;
  void* stage2 = nullptr;                 // second staging state: gbs_step_host_stream alternates
  cudaStream_t copy_stream = nullptr;     // gbs_step_host_stream: host-to-device copies
  cudaStream_t d2h_stream = nullptr;      // and device-to-host copies (separate copy engines)
  cudaEvent_t ev_in[2] = {}, ev_out[2] = {}, ev_d2h[2] = {};
  void* levels = nullptr;
  void* ds_y0 = nullptr;                  // GBS_F32X2: y_in, kappa, b as FP32 pairs
  void* ds_kappa = nullptr;
  void* ds_b = nullptr;
  int levels_steps = 0;
  void* mu0 = nullptr;
  void* mu1 = nullptr;
  void* mu_shared = nullptr;
  float2* gpair = nullptr;                // FP32 path: per-sequence gradient sums as (hi, lo) pairs
  FusedWork* fw = nullptr;                // time-blocked path: schedule and level store
  bool fw_ready = false;
  Tb3Work* tb3 = nullptr;                 // 3D time-blocked passes: tiles and second level pair
  bool tb3_ready = false;
  // sequence-fused one-level steps (FP32 2D/3D acoustics on the one-level kernels): a level pair
  // per sequence, and the tensor map over all of them
  void* Lms = nullptr;
  int64_t Lms_elems = 0;
  bool ms_ready = false;
  bool ms_tma = false;
  alignas(64) unsigned char ms_tmap[128] = {};
  int opt_seqfuse = -1;                   // -1: by dimension (2D on; 3D off, measured slower on GB300)
  int opt_seqgroup = -1;                  // most sequences per fused launch: -1 = by dimension
  // execution
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  int opt_kernel = GBS_KERNEL_AUTO;
  int opt_graph = 1;
  int opt_check_stability = 0;
  int opt_time_kernels = 0;
  int opt_hseg = 256;
  int opt_zseg = 128;                     // 3D time-blocked passes: z-planes per block
  int opt_tmax = 0;                       // 0: the kernel's largest pass depth
  int opt_schedule = 0;
  int opt_tma = -1;                       // tensor-map staging of the FP32 tiled step: -1 where measured
                                          // faster (3D), 1 wherever available, 0 off
  bool tma_ok = false;                    // lf_tmap holds the maps of L0 and L1
  alignas(64) unsigned char lf_tmap[2][128] = {};
  int64_t opt_spin_limit = 1 << 20;
  int opt_inject_wait = 0;
  uint32_t fused_mask = ~0u;              // sequences of the prepared time-blocked schedule
  int opt_combine = 0;                    // time-blocked FP32 path: 0 = FP64 combine, 1 = compensated
                                          // FP32 pairs
  std::vector<cudaEvent_t> tev;           // event pairs for kernel timing
  std::vector<double> tev_bytes;
  int tev_used = 0;
  std::vector<int64_t> active_pts;        // points updated by plain step (k, n)
  uint64_t sched_version = 1;
  std::vector<GraphEntry> graphs;
  int64_t launches = 0;
  std::string err;
};

namespace {

gbs_status fail(gbs_ctx* h, gbs_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (h) h->err = buf;
  else g_create_error = buf;
  return st;
}

#define CK(h, call)                                                                                 \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) return fail((h), GBS_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

int fields_of(int system, int ndim) {
  return system == GBS_WAVE1D ? 2 : system == GBS_ONEWAY_SPECTRAL ? 1 : 1 + ndim;
}

double symbol_max(int R) {
  // max over theta of |sum_j a_j 2 sin(j theta)| -- sampled densely, then refined
  auto s = [R](double t) {
    return R == 2 ? (2.0 * (2.0 / 3.0) * std::sin(t) - 2.0 * (1.0 / 12.0) * std::sin(2 * t))
                  : (2.0 * 0.75 * std::sin(t) - 2.0 * 0.15 * std::sin(2 * t) + 2.0 * (1.0 / 60.0) * std::sin(3 * t));
  };
  double best = 0, bt = 0;
  const int n = 20000;
  for (int i = 0; i <= n; ++i) {
    const double t = M_PI * i / n;
    if (std::fabs(s(t)) > best) best = std::fabs(s(t)), bt = t;
  }
  double lo = std::max(0.0, bt - M_PI / n), hi = std::min(M_PI, bt + M_PI / n);
  for (int it = 0; it < 200; ++it) {
    const double m1 = lo + (hi - lo) / 3, m2 = hi - (hi - lo) / 3;
    if (std::fabs(s(m1)) < std::fabs(s(m2))) lo = m1;
    else hi = m2;
  }
  return std::fabs(s(0.5 * (lo + hi)));
}

gbs_status validate_problem(const gbs_problem* pb, gbs_ctx* h) {
  if (!pb) return fail(h, GBS_ERR_INVALID, "problem description is NULL");
  if (pb->system != GBS_WAVE1D && pb->system != GBS_ACOUSTIC && pb->system != GBS_ONEWAY_SPECTRAL)
    return fail(h, GBS_ERR_INVALID, "system must be GBS_WAVE1D, GBS_ACOUSTIC or GBS_ONEWAY_SPECTRAL");
  if (pb->system != GBS_ACOUSTIC && pb->ndim != 1) return fail(h, GBS_ERR_INVALID, "this system needs ndim == 1");
  if (pb->ndim < 1 || pb->ndim > 3) return fail(h, GBS_ERR_INVALID, "ndim must be 1, 2 or 3");
  if (pb->system == GBS_ONEWAY_SPECTRAL) {
    if (pb->fd_order != 0) return fail(h, GBS_ERR_INVALID, "GBS_ONEWAY_SPECTRAL takes fd_order = 0 (spectral)");
    if (pb->precision != GBS_F64) return fail(h, GBS_ERR_INVALID, "GBS_ONEWAY_SPECTRAL runs in GBS_F64");
    for (int p = 0; p < pb->batch && pb->shape; ++p) {
      const int64_t n = pb->shape[3 * p];
      if (n < 8 || n > kSpectralMaxN || (n & (n - 1)))
        return fail(h, GBS_ERR_INVALID, "problem %d: spectral size must be a power of two in [8, %d]", p, kSpectralMaxN);
    }
  } else if (pb->fd_order != 4 && pb->fd_order != 6) {
    return fail(h, GBS_ERR_INVALID, "fd_order must be 4 or 6");
  }
  if (pb->precision != GBS_F32_STATE_F64_COMBINE && pb->precision != GBS_F64 && pb->precision != GBS_F32X2)
    return fail(h, GBS_ERR_INVALID, "unknown precision");
  if (pb->batch < 1) return fail(h, GBS_ERR_INVALID, "batch must be >= 1");
  if (!pb->shape || !pb->dx) return fail(h, GBS_ERR_INVALID, "shape and dx arrays are required");
  if (pb->enable_adjoint && pb->system != GBS_ACOUSTIC)
    return fail(h, GBS_ERR_INVALID, "the adjoint is provided for GBS_ACOUSTIC only");
  const int R = pb->fd_order / 2;
  for (int p = 0; p < pb->batch; ++p) {
    for (int d = 0; d < 3; ++d) {
      const int64_t n = pb->shape[3 * p + d];
      if (d < pb->ndim) {
        if (n < R || n > (int64_t(1) << 30))
          return fail(h, GBS_ERR_INVALID, "problem %d: size %lld along dim %d outside [%d, 2^30]", p, (long long)n, d, R);
        const double dx = pb->dx[3 * p + d];
        if (!(dx > 0) || !std::isfinite(dx)) return fail(h, GBS_ERR_INVALID, "problem %d: dx[%d] must be > 0", p, d);
      } else if (n != 1) {
        return fail(h, GBS_ERR_INVALID, "problem %d: unused dim %d must have size 1", p, d);
      }
    }
    if (pb->shape[3 * p] * pb->shape[3 * p + 1] * pb->shape[3 * p + 2] >= (int64_t(1) << 31))
      return fail(h, GBS_ERR_INVALID, "problem %d has 2^31 or more grid points", p);
  }
  return GBS_OK;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class T>
gbs_status dalloc(gbs_ctx* h, T** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return GBS_OK;
  if (cudaMalloc(reinterpret_cast<void**>(p), bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(h, GBS_ERR_NOMEM, "cudaMalloc of %zu bytes failed", bytes);
  }
  return GBS_OK;
}

void free_graphs(gbs_ctx* h) {
  for (auto& g : h->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  h->graphs.clear();
}

void free_all(gbs_ctx* h) {
  free_graphs(h);
  void* ptrs[] = {h->b, h->d_probs, h->d_slots, h->d_H, h->d_hk, h->d_hkf, h->d_hkq, h->d_err, h->d_red, h->d_cmax, h->f0, h->L0, h->L1,
                  h->acc, h->stage, h->stage2, h->levels, h->mu0, h->mu1, h->mu_shared, h->ds_y0, h->ds_kappa,
                  h->ds_b, h->gpair};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  if (h->d2h_stream) cudaStreamDestroy(h->d2h_stream);
  for (int i = 0; i < 2; ++i) {
    if (h->ev_in[i]) cudaEventDestroy(h->ev_in[i]);
    if (h->ev_out[i]) cudaEventDestroy(h->ev_out[i]);
    if (h->ev_d2h[i]) cudaEventDestroy(h->ev_d2h[i]);
  }
  for (cudaEvent_t e : h->tev) cudaEventDestroy(e);
  h->tev.clear();
  fused_destroy(h->fw);
  h->fw = nullptr;
  tb3_destroy(h->tb3);
  h->tb3 = nullptr;
  if (h->Lms) cudaFree(h->Lms);
  h->Lms = nullptr;
}

struct Sizes {
  int64_t state_elems = 0, media_elems = 0;
};

Sizes sizes_of(const gbs_problem* pb) {
  Sizes s;
  const int F = fields_of(pb->system, pb->ndim);
  for (int p = 0; p < pb->batch; ++p) {
    const int64_t pts = pb->shape[3 * p] * pb->shape[3 * p + 1] * pb->shape[3 * p + 2];
    s.state_elems += F * pts;
    s.media_elems += pts;
  }
  return s;
}

// ---------------------------------------------------------------------------
// Scheme set-up
// ---------------------------------------------------------------------------

// Dual Vandermonde system sum_i z_i x_i^j = r_j (j = 0..n) by Bjorck-Pereyra, in dd.
// |R(iy)|^2 - 1 for the scheme; R = sum_k c_k P_k(iy), P_k from the GBS recurrence on y' = lambda y.
double abs2_minus_one(const Slot& s, double y) {
  std::complex<double> R = 0;
  for (int k = 0; k < s.m; ++k) {
    const int N = s.steps[k];
    const std::complex<double> z(0.0, y / N);
    std::complex<double> y_prev = 1.0, y_cur = 1.0 + z;  // y_0, y_1 (Forward Euler)
    std::complex<double> y_before = y_prev;
    for (int j = 1; j <= N; ++j) {                        // leap-frog
      const std::complex<double> y_next = y_prev + 2.0 * z * y_cur;
      y_before = y_prev;
      y_prev = y_cur;
      y_cur = y_next;
    }
    // y_before = y_(N-1), y_prev = y_N, y_cur = y_(N+1)
    R += s.c[k] * (y_before + 2.0 * y_prev + y_cur) * 0.25;
  }
  return std::norm(R) - 1.0;
}

double scan_isb(const Slot& s) {
  int nmax = 0;
  for (int k = 0; k < s.m; ++k) nmax = std::max(nmax, s.steps[k]);
  const double ymax = 1.5 * (nmax + 1);  // ISB_n <= 1 for explicit methods
  const double dy = 1e-3;
  const double tol = 1e-12;
  double prev = 0.0;
  for (double y = dy; y <= ymax; y += dy) {
    if (abs2_minus_one(s, y) > tol) {
      double lo = prev, hi = y;
      for (int it = 0; it < 80; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (abs2_minus_one(s, mid) > tol) hi = mid;
        else lo = mid;
      }
      return lo;
    }
    prev = y;
  }
  return ymax;
}

gbs_status prepare_fused(gbs_ctx* h);

// h_k = H_p / N_k for every problem and sequence, computed once on the host so that no
// kernel divides in FP64 (GB300's FP64 rate is low).
gbs_status upload_hk(gbs_ctx* h) {
  if ((int)h->cur_H.size() != h->batch) return GBS_OK;
  h->hk_host.assign((size_t)h->batch * GBS_MAX_SEQ, 0.0);
  h->hkf_host.assign((size_t)h->batch * GBS_MAX_SEQ, make_float2(0.f, 0.f));
  h->hkq_host.assign((size_t)h->batch * GBS_MAX_SEQ, make_float4(0.f, 0.f, 0.f, 0.f));
  for (int p = 0; p < h->batch; ++p) {
    const Slot& s = h->slots[h->slot_of[p]];
    for (int k = 0; k < s.m; ++k) {
      const double hk = h->cur_H[p] / s.steps[k];
      h->hk_host[(size_t)p * GBS_MAX_SEQ + k] = hk;
      h->hkf_host[(size_t)p * GBS_MAX_SEQ + k] = make_float2((float)hk, (float)(2.0 * hk));
      h->hkq_host[(size_t)p * GBS_MAX_SEQ + k] = fp32_step_consts(h->probs[p], hk, h->R);
    }
  }
  CK(h, cudaMemcpyAsync(h->d_hk, h->hk_host.data(), sizeof(double) * h->hk_host.size(), cudaMemcpyHostToDevice,
                        h->stream));
  CK(h, cudaMemcpyAsync(h->d_hkf, h->hkf_host.data(), sizeof(float2) * h->hkf_host.size(), cudaMemcpyHostToDevice,
                        h->stream));
  CK(h, cudaMemcpyAsync(h->d_hkq, h->hkq_host.data(), sizeof(float4) * h->hkq_host.size(), cudaMemcpyHostToDevice,
                        h->stream));
  return GBS_OK;
}

gbs_status upload_slots(gbs_ctx* h) {
  SlotDev sd[GBS_MAX_SLOTS];
  std::memset(sd, 0, sizeof sd);
  for (int i = 0; i < GBS_MAX_SLOTS; ++i) {
    sd[i].m = h->slots[i].m;
    for (int k = 0; k < h->slots[i].m; ++k) {
      sd[i].steps[k] = h->slots[i].steps[k];
      sd[i].c[k] = h->slots[i].c[k];
    }
    split_weights(sd[i]);
  }
  CK(h, cudaStreamSynchronize(h->stream));
  CK(h, cudaMemcpy(h->d_slots, sd, sizeof sd, cudaMemcpyHostToDevice));
  for (int p = 0; p < h->batch; ++p) h->probs[p].slot = h->slot_of[p];
  CK(h, cudaMemcpy(h->d_probs, h->probs.data(), sizeof(ProbDev) * h->batch, cudaMemcpyHostToDevice));
  ++h->sched_version;
  gbs_status st = upload_hk(h);
  if (st != GBS_OK) return st;
  return prepare_fused(h);
}

// Tensor-map staging of the FP32 tiled step: on request, or by default in 3D, where it measured
// faster than load staging (512^3: 94.8 against 90.1 G updates/s; 2D 2048^2: 109.8 against 110.6).
bool tma_in_use(const gbs_ctx* h) { return h->tma_ok && (h->opt_tma == 1 || (h->opt_tma < 0 && h->ndim == 3)); }

gbs_status build_plan(gbs_ctx* h, StepPlan* p) {
  std::memset(p, 0, sizeof *p);
  p->system = h->system;
  p->ndim = h->ndim;
  p->R = h->R;
  p->f64 = h->f64;
  p->ds = h->ds;
  p->ds_y0 = h->ds_y0;
  p->ds_kappa = h->ds_kappa;
  p->ds_b = h->ds_b;
  p->probs_media_elems = h->media_elems;
  for (const ProbDev& q : h->probs) p->max_nx = std::max<int64_t>(p->max_nx, q.n[0]);
  p->nx_vec = 1;
  for (const ProbDev& q : h->probs) p->nx_vec &= (q.n[0] % 4 == 0) ? 1 : 0;
  p->F = h->F;
  p->batch = h->batch;
  p->probs = h->d_probs;
  p->slots = h->d_slots;
  p->H = h->d_H;
  p->hk = h->d_hk;
  p->hkf = h->d_hkf;
  p->hkq = h->d_hkq;
  p->total_blocks = h->total_blocks;
  p->total_tiles = h->total_tiles;
  p->state_elems = h->state_elems;
  p->kappa = h->kappa;
  p->b = h->b;
  p->f0 = h->f0;
  p->L0 = h->L0;
  p->L1 = h->L1;
  p->acc = h->acc;
  p->err = h->d_err;
  p->seq_mask = ~0u;
  p->partial = 0;
  if (tma_in_use(h)) {
    p->lf_tmap[0] = h->lf_tmap[0];
    p->lf_tmap[1] = h->lf_tmap[1];
  }
  h->active_pts.assign((size_t)GBS_MAX_SEQ * (GBS_MAX_STEPS + 1), 0);
  for (int q = 0; q < h->batch; ++q) {
    const Slot& s = h->slots[h->slot_of[q]];
    if (!s.set) return fail(h, GBS_ERR_STATE, "problem %d uses weight slot %d which has no weights", q, h->slot_of[q]);
    p->max_m = std::max(p->max_m, s.m);
    for (int k = 0; k < s.m; ++k) {
      p->max_steps_k[k] = std::max(p->max_steps_k[k], s.steps[k]);
      for (int n = 1; n <= s.steps[k]; ++n) h->active_pts[k * (GBS_MAX_STEPS + 1) + n] += h->probs[q].pts;
    }
  }
  p->active_pts = h->active_pts.data();
  // plain leap-frog step: read y_(n-1) and y_n, write y_(n+1) (F fields each), read the media,
  // and FP32 states (increment form) read f0
  p->unit_bytes = (double)h->esz * (3.0 * h->F + (h->system == GBS_ACOUSTIC ? 2.0 : 0.0) +
                                    (h->esz == 4 && !h->ds ? h->F : 0.0));
  // adjoint reverse step: read M[j+1] and M[j+2], write M[j] (F fields each), the media, the
  // forward level's velocities (divergence for the gradient), FP64 gradient read and write
  p->adj_unit_bytes = (double)h->esz * (3.0 * h->F + 2.0 + h->ndim) + 16.0;
  if (h->opt_time_kernels) {
    p->tev = h->tev.data();
    p->tev_bytes = h->tev_bytes.data();
    p->tev_cap = (int)h->tev.size() / 2;
    p->tev_used = &h->tev_used;
  }
  return GBS_OK;
}

gbs_status prepare_time_blocked(gbs_ctx* h);

// The sequence-fused one-level step's level pairs (set-up time: may allocate), where the
// one-level kernels run FP32 2D/3D acoustics; without the memory for them the step runs one
// sequence per launch.
gbs_status prepare_seqfuse(gbs_ctx* h) {
  const bool was = h->ms_ready;
  h->ms_ready = false;
  const bool want = h->opt_seqfuse > 0 || (h->opt_seqfuse < 0 && h->ndim == 2);
  bool applies = want && h->system == GBS_ACOUSTIC && h->ndim >= 2 && h->esz == 4 && !h->ds &&
                 !h->f64 && !(h->opt_kernel != GBS_KERNEL_PLAIN && (h->fw_ready || h->tb3_ready));
  for (int i = 0; i < GBS_MAX_SLOTS && applies; ++i)   // distinct step counts within every slot
    for (int a = 0; a < h->slots[i].m && applies; ++a)
      for (int b = a + 1; b < h->slots[i].m; ++b)
        if (h->slots[i].steps[a] == h->slots[i].steps[b]) applies = false;
  StepPlan p;
  if (!applies || build_plan(h, &p) != GBS_OK) {
    h->err.clear();
    if (h->Lms && !applies) {
      CK(h, cudaStreamSynchronize(h->stream));
      cudaFree(h->Lms);
      h->Lms = nullptr;
      h->Lms_elems = 0;
    }
    if (was) ++h->sched_version;
    return GBS_OK;
  }
  const int64_t need = 2 * (int64_t)p.max_m * h->state_elems;
  if (h->Lms_elems < need) {
    CK(h, cudaStreamSynchronize(h->stream));
    if (h->Lms) cudaFree(h->Lms);
    h->Lms = nullptr;
    h->Lms_elems = 0;
    if (cudaMalloc(&h->Lms, sizeof(float) * (size_t)need) != cudaSuccess) {
      cudaGetLastError();   // not enough memory: one sequence per launch
      h->Lms = nullptr;
      ++h->sched_version;
      return GBS_OK;
    }
    h->Lms_elems = need;
  }
  h->ms_tma = false;
  if (h->batch == 1 && h->probs[0].n[0] % 4 == 0) {
    const ProbDev& q = h->probs[0];
    h->ms_tma = lf_tma_encode(h->ms_tmap, h->Lms, (int)q.n[0], (int)q.n[1], (int)q.n[2], h->F * 2 * p.max_m, h->R) == 0;
  }
  h->ms_ready = true;
  ++h->sched_version;
  return GBS_OK;
}

gbs_status prepare_fused(gbs_ctx* h) {
  gbs_status st = prepare_time_blocked(h);
  if (st != GBS_OK) return st;
  return prepare_seqfuse(h);
}

// (Re)build the time-blocked schedule when it applies (set-up time: may allocate).
gbs_status prepare_time_blocked(gbs_ctx* h) {
  h->fw_ready = false;
  h->tb3_ready = false;
  if (h->opt_kernel == GBS_KERNEL_PLAIN) return GBS_OK;
  StepPlan p;
  if (build_plan(h, &p) != GBS_OK) {  // some slot without weights yet: nothing to prepare
    h->err.clear();
    return GBS_OK;
  }
  SlotDev sd[GBS_MAX_SLOTS];
  std::memset(sd, 0, sizeof sd);
  for (int i = 0; i < GBS_MAX_SLOTS; ++i) {
    sd[i].m = h->slots[i].m;
    for (int k = 0; k < h->slots[i].m; ++k) {
      sd[i].steps[k] = h->slots[i].steps[k];
      sd[i].c[k] = h->slots[i].c[k];
    }
    split_weights(sd[i]);
  }
  char msg[256] = {0};
  // 3D: the pass kernel only when asked for (GBS_KERNEL_FUSED); under GBS_KERNEL_AUTO the
  // one-level kernel, measured faster on GB300
  if (tb3_supported(p, h->probs.data(), sd, GBS_MAX_SLOTS)) {
    if (h->opt_kernel != GBS_KERNEL_FUSED) return GBS_OK;
    CK(h, cudaStreamSynchronize(h->stream));
    const int r = tb3_prepare(h->tb3, p, h->probs.data(), sd, h->opt_zseg, msg, sizeof msg);
    if (r == -2) return fail(h, GBS_ERR_NOMEM, "%s", msg);
    if (r < 0) return fail(h, GBS_ERR_CUDA, "%s", msg);
    h->tb3_ready = true;
    ++h->sched_version;
    return GBS_OK;
  }
  if (!fused_supported(p, h->probs.data())) return GBS_OK;
  CK(h, cudaStreamSynchronize(h->stream));
  const FusedTune tune{h->opt_hseg, h->opt_tmax ? h->opt_tmax : fused_max_levels(), h->opt_schedule, h->fused_mask};
  const int r = fused_prepare(h->fw, p, h->probs.data(), sd, tune, msg, sizeof msg);
  if (r == -2) return fail(h, GBS_ERR_NOMEM, "%s", msg);
  if (r < 0) return fail(h, GBS_ERR_CUDA, "%s", msg);
  h->fw_ready = true;
  ++h->sched_version;
  return GBS_OK;
}

gbs_status set_H(gbs_ctx* h, const double* H) {
  bool same = (int)h->cur_H.size() == h->batch;
  for (int p = 0; p < h->batch; ++p) {
    if (!(H[p] > 0) || !std::isfinite(H[p])) return fail(h, GBS_ERR_INVALID, "H[%d] must be finite and > 0", p);
    if (same && h->cur_H[p] != H[p]) same = false;
  }
  if (same) return GBS_OK;
  h->cur_H.assign(H, H + h->batch);
  // pageable source: the call returns once the values are staged, so cur_H may change afterwards
  CK(h, cudaMemcpyAsync(h->d_H, h->cur_H.data(), sizeof(double) * h->batch, cudaMemcpyHostToDevice, h->stream));
  return upload_hk(h);
}

// Sequences per fused launch in 3D, where each launch's z-neighbour planes stay in the cache
// only while the group is small.
constexpr int kSeqGroup3D = 4;

// The one-level path: sequence-fused where its level pairs are ready.
int plain_step(gbs_ctx* h, const StepPlan& p, const void* yi, void* yo, cudaStream_t s) {
  if (!h->ms_ready) return plain_macro_step(p, yi, yo, s);
  const bool map = h->ms_tma && (h->opt_tma == 1 || (h->opt_tma < 0 && h->ndim == 3));
  const int group = h->opt_seqgroup >= 0 ? h->opt_seqgroup : h->ndim == 3 ? kSeqGroup3D : 0;
  const SeqLevels lv{h->Lms, h->state_elems, map ? h->ms_tmap : nullptr, group};
  return plain_macro_step_seqfused(p, lv, yi, yo, s);
}

bool use_fused(gbs_ctx* h, const StepPlan&) {
  return h->opt_kernel != GBS_KERNEL_PLAIN && (h->fw_ready || h->tb3_ready);
}

// Enqueue one macro-step on stream s (no graph).  Returns launches or -1.
int enqueue_macro(gbs_ctx* h, const StepPlan& p, const void* yi, void* yo, cudaStream_t s, int kernel) {
  if (kernel == GBS_KERNEL_FUSED && h->tb3_ready) return tb3_macro_step(h->tb3, p, yi, yo, s);
  if (kernel == GBS_KERNEL_FUSED) return fused_macro_step(h->fw, p, yi, yo, s, h->d_err);
  return plain_step(h, p, yi, yo, s);
}

gbs_status run_macro(gbs_ctx* h, const StepPlan& p, const void* yi, void* yo) {
  const int kernel = use_fused(h, p) ? GBS_KERNEL_FUSED : GBS_KERNEL_PLAIN;
  if (!h->opt_graph || h->opt_time_kernels) {
    const int n = enqueue_macro(h, p, yi, yo, h->stream, kernel);
    if (n < 0) return fail(h, GBS_ERR_CUDA, "kernel launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    h->launches += n;
    return GBS_OK;
  }
  GraphEntry* ge = nullptr;
  for (auto& g : h->graphs)
    if (g.yi == yi && g.yo == yo && g.kernel == kernel && g.version == h->sched_version) ge = &g;
  if (!ge) {
    if (h->graphs.size() >= 4) {
      cudaGraphExecDestroy(h->graphs.front().exec);
      h->graphs.erase(h->graphs.begin());
    }
    GraphEntry g;
    g.yi = yi;
    g.yo = yo;
    g.kernel = kernel;
    g.version = h->sched_version;
    CK(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    const int n = enqueue_macro(h, p, yi, yo, h->cap, kernel);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->cap, &graph);
    if (n < 0 || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return fail(h, GBS_ERR_CUDA, "graph capture of the macro-step failed");
    }
    const cudaError_t e2 = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e2 != cudaSuccess) return fail(h, GBS_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e2));
    g.launches = n;
    h->graphs.push_back(g);
    ge = &h->graphs.back();
  }
  CK(h, cudaGraphLaunch(ge->exec, h->stream));
  h->launches += ge->launches;
  return GBS_OK;
}

}  // namespace

// ===========================================================================
// Public entry points
// ===========================================================================

extern "C" {

size_t gbs_state_elems(const gbs_problem* pb) {
  if (validate_problem(pb, nullptr) != GBS_OK) return 0;
  return (size_t)sizes_of(pb).state_elems;
}

size_t gbs_workspace_bytes(const gbs_problem* pb, int max_steps) {
  if (validate_problem(pb, nullptr) != GBS_OK || max_steps < 0) return 0;
  const Sizes s = sizes_of(pb);
  const size_t esz = pb->precision == GBS_F32_STATE_F64_COMBINE ? 4 : 8;
  size_t bytes = 0;
  bytes += 5 * s.state_elems * esz;       // f0, L0, L1, two staging states
  bytes += 8 * s.state_elems;             // acc
  bytes += s.media_elems * esz;           // b
  if (pb->precision == GBS_F32X2) bytes += 8 * (s.state_elems + 2 * s.media_elems);   // pair copies
  if (pb->system == GBS_ACOUSTIC && pb->ndim == 3 && pb->precision == GBS_F32_STATE_F64_COMBINE)
    bytes += tb3_workspace_bytes(s.state_elems);   // the 3D time-blocked passes' second level pair
  if (pb->enable_adjoint) {
    bytes += (size_t)(max_steps + 2 + 3) * s.state_elems * esz;
    if (pb->precision == GBS_F32_STATE_F64_COMBINE) bytes += 8 * s.media_elems;   // gradient pairs
  }
  bytes += sizeof(ProbDev) * pb->batch + sizeof(SlotDev) * GBS_MAX_SLOTS + 8 * pb->batch * 2 +
           8 * (4 * kNormBlocks + 4) + 64;
  return bytes;
}

gbs_status gbs_create(const gbs_problem* pb, const void* kappa, const void* rho, void* cuda_stream,
                      gbs_handle* out) {
  g_create_error.clear();
  if (!out) return fail(nullptr, GBS_ERR_INVALID, "out pointer is NULL");
  *out = nullptr;
  gbs_status st = validate_problem(pb, nullptr);
  if (st != GBS_OK) return st;
  if (pb->system != GBS_ACOUSTIC && (kappa || rho))
    return fail(nullptr, GBS_ERR_INVALID, "only GBS_ACOUSTIC takes media (kappa and rho must be NULL)");
  if (pb->system == GBS_ACOUSTIC && (!is_device_ptr(kappa) || !is_device_ptr(rho)))
    return fail(nullptr, GBS_ERR_INVALID, "kappa and rho must be device pointers");
  gbs_ctx* h = new gbs_ctx();
  h->system = pb->system;
  h->ndim = pb->ndim;
  h->order = pb->fd_order;
  h->R = pb->fd_order / 2;
  h->f64 = pb->precision != GBS_F32_STATE_F64_COMBINE;   // FP64 states and media in the API
  h->ds = pb->precision == GBS_F32X2;
  h->esz = h->f64 ? 8 : 4;
  h->batch = pb->batch;
  h->F = fields_of(pb->system, pb->ndim);
  h->adjoint = pb->enable_adjoint != 0;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->slot_of.assign(h->batch, 0);
  h->probs.resize(h->batch);
  int64_t soff = 0, moff = 0, blk = 0;
  for (int p = 0; p < h->batch; ++p) {
    ProbDev& q = h->probs[p];
    std::memset(&q, 0, sizeof q);
    for (int d = 0; d < 3; ++d) {
      q.n[d] = (int)pb->shape[3 * p + d];
      q.inv_dx[d] = d < h->ndim ? 1.0 / pb->dx[3 * p + d] : 0.0;
    }
    fill_fp32_consts(q, h->ndim, h->R);
    q.pts = (int64_t)q.n[0] * q.n[1] * q.n[2];
    q.state_off = soff;
    q.media_off = moff;
    q.blk_begin = blk;
    soff += h->F * q.pts;
    moff += q.pts;
    blk += (q.pts + kPlainBlock - 1) / kPlainBlock;
  }
  h->state_elems = soff;
  h->media_elems = moff;
  h->total_blocks = blk;
  h->total_tiles = assign_tiles(h->probs.data(), h->batch, h->ndim);
  if (blk > 0x7fffffff) {
    delete h;
    return fail(nullptr, GBS_ERR_INVALID, "problem too large for one launch grid");
  }
  auto bail = [&](gbs_status s) {
    g_create_error = h->err;
    free_all(h);
    delete h;
    return s;
  };
  const size_t E = (size_t)h->state_elems, P = (size_t)h->media_elems;
  if ((st = dalloc(h, &h->d_probs, sizeof(ProbDev) * h->batch)) != GBS_OK) return bail(st);
  if ((st = dalloc(h, &h->d_slots, sizeof(SlotDev) * GBS_MAX_SLOTS)) != GBS_OK) return bail(st);
  if ((st = dalloc(h, &h->d_H, sizeof(double) * h->batch)) != GBS_OK) return bail(st);
  if ((st = dalloc(h, &h->d_hk, sizeof(double) * h->batch * GBS_MAX_SEQ)) != GBS_OK) return bail(st);
  if ((st = dalloc(h, &h->d_hkf, sizeof(float2) * h->batch * GBS_MAX_SEQ)) != GBS_OK) return bail(st);
  if ((st = dalloc(h, &h->d_hkq, sizeof(float4) * h->batch * GBS_MAX_SEQ)) != GBS_OK) return bail(st);
  if ((st = dalloc(h, &h->d_err, 64)) != GBS_OK) return bail(st);
  if ((st = dalloc(h, &h->d_red, sizeof(double) * (4 * kNormBlocks + 4))) != GBS_OK) return bail(st);
  if ((st = dalloc(h, &h->d_cmax, sizeof(double) * h->batch)) != GBS_OK) return bail(st);
  if ((st = dalloc(h, &h->f0, E * h->esz)) != GBS_OK) return bail(st);
  if ((st = dalloc(h, &h->L0, E * h->esz)) != GBS_OK) return bail(st);
  if ((st = dalloc(h, &h->L1, E * h->esz)) != GBS_OK) return bail(st);
  if ((st = dalloc(h, &h->acc, E * sizeof(double))) != GBS_OK) return bail(st);
  if ((st = dalloc(h, &h->stage, E * h->esz)) != GBS_OK) return bail(st);
  if ((st = dalloc(h, &h->stage2, E * h->esz)) != GBS_OK) return bail(st);
  if (h->system == GBS_ACOUSTIC && (st = dalloc(h, &h->b, P * h->esz)) != GBS_OK) return bail(st);
  if (h->ds) {   // FP32 pairs take 8 bytes, like the FP64 values they are made from
    if ((st = dalloc(h, &h->ds_y0, E * 8)) != GBS_OK) return bail(st);
    if (h->system == GBS_ACOUSTIC && ((st = dalloc(h, &h->ds_kappa, P * 8)) != GBS_OK ||
                                      (st = dalloc(h, &h->ds_b, P * 8)) != GBS_OK))
      return bail(st);
  }
  if (h->adjoint) {
    if ((st = dalloc(h, &h->mu0, E * h->esz)) != GBS_OK) return bail(st);
    if ((st = dalloc(h, &h->mu1, E * h->esz)) != GBS_OK) return bail(st);
    if ((st = dalloc(h, &h->mu_shared, E * h->esz)) != GBS_OK) return bail(st);
    if (!h->f64 && (st = dalloc(h, &h->gpair, P * sizeof(float2))) != GBS_OK) return bail(st);
  }
  if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->d2h_stream, cudaStreamNonBlocking) != cudaSuccess) {
    fail(h, GBS_ERR_CUDA, "cudaStreamCreate failed");
    return bail(GBS_ERR_CUDA);
  }
  for (int i = 0; i < 2; ++i)
    if (cudaEventCreateWithFlags(&h->ev_in[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_out[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_d2h[i], cudaEventDisableTiming) != cudaSuccess) {
      fail(h, GBS_ERR_CUDA, "cudaEventCreate failed");
      return bail(GBS_ERR_CUDA);
    }
  if (cudaMemset(h->d_err, 0, 64) != cudaSuccess || cudaMemset(h->d_slots, 0, sizeof(SlotDev) * GBS_MAX_SLOTS) != cudaSuccess ||
      cudaMemcpy(h->d_probs, h->probs.data(), sizeof(ProbDev) * h->batch, cudaMemcpyHostToDevice) != cudaSuccess) {
    fail(h, GBS_ERR_CUDA, "workspace initialisation failed");
    return bail(GBS_ERR_CUDA);
  }
  h->cmax.assign(h->batch, 1.0);
  // tensor maps of the two level buffers for the FP32 tiled step (one 2D/3D acoustic problem,
  // nx a multiple of 4); without them the kernel stages with loads
  if (h->system == GBS_ACOUSTIC && h->ndim >= 2 && h->batch == 1 && h->esz == 4 && !h->ds && !h->f64 &&
      h->probs[0].n[0] % 4 == 0) {
    const ProbDev& q = h->probs[0];
    h->tma_ok = lf_tma_encode(h->lf_tmap[0], h->L0, (int)q.n[0], (int)q.n[1], (int)q.n[2], h->F, h->R) == 0 &&
                lf_tma_encode(h->lf_tmap[1], h->L1, (int)q.n[0], (int)q.n[1], (int)q.n[2], h->F, h->R) == 0;
  }
  h->fw = fused_create();
  h->tb3 = tb3_create();
  if (h->system == GBS_ONEWAY_SPECTRAL && spectral_setup() < 0) {
    fail(h, GBS_ERR_CUDA, "the spectral kernel cannot get its shared memory");
    return bail(GBS_ERR_CUDA);
  }
  *out = h;
  if (h->system == GBS_ACOUSTIC) {
    st = gbs_set_media(h, kappa, rho);
    if (st != GBS_OK) {
      g_create_error = h->err;
      *out = nullptr;
      free_all(h);
      delete h;
      return st;
    }
  }
  return GBS_OK;
}

gbs_status gbs_set_media(gbs_handle h, const void* kappa, const void* rho) {
  if (!h) return fail(nullptr, GBS_ERR_INVALID, "handle is NULL");
  if (h->system != GBS_ACOUSTIC) return fail(h, GBS_ERR_INVALID, "media apply to GBS_ACOUSTIC only");
  if (!is_device_ptr(kappa) || !is_device_ptr(rho)) return fail(h, GBS_ERR_INVALID, "kappa and rho must be device pointers");
  h->kappa = kappa;
  if (prep_media(h->f64, rho, h->b, h->media_elems, h->stream) < 0)
    return fail(h, GBS_ERR_CUDA, "media preparation failed: %s", cudaGetErrorString(cudaGetLastError()));
  if (media_cmax(h->f64, kappa, h->b, h->d_probs, h->batch, h->d_cmax, h->stream) < 0)
    return fail(h, GBS_ERR_CUDA, "media reduction failed: %s", cudaGetErrorString(cudaGetLastError()));
  CK(h, cudaStreamSynchronize(h->stream));
  CK(h, cudaMemcpy(h->cmax.data(), h->d_cmax, sizeof(double) * h->batch, cudaMemcpyDeviceToHost));
  for (int p = 0; p < h->batch; ++p)
    if (!(h->cmax[p] > 0) || !std::isfinite(h->cmax[p]))
      return fail(h, GBS_ERR_NONFINITE, "problem %d: media give a non-positive or non-finite wave speed", p);
  ++h->sched_version;  // graphs hold the kappa pointer
  return GBS_OK;
}

gbs_status gbs_set_weights(gbs_handle h, int slot, int order_p, int n_dep, const int* steps_dep, int n_free,
                           const int* steps_free, const double* c_free, const double* c_full) {
  if (!h) return fail(nullptr, GBS_ERR_INVALID, "handle is NULL");
  if (slot < 0 || slot >= GBS_MAX_SLOTS) return fail(h, GBS_ERR_INVALID, "slot %d out of range", slot);
  if (order_p < 2 || order_p % 2) return fail(h, GBS_ERR_INVALID, "order must be even and >= 2");
  if (n_dep != order_p / 2) return fail(h, GBS_ERR_INVALID, "n_dep must equal order/2 (%d)", order_p / 2);
  if (n_free < 0 || n_dep + n_free > GBS_MAX_SEQ) return fail(h, GBS_ERR_INVALID, "too many sequences (max %d)", GBS_MAX_SEQ);
  if (!steps_dep || (n_free > 0 && !steps_free)) return fail(h, GBS_ERR_INVALID, "step count arrays are required");
  if (n_free > 0 && !c_free && !c_full) return fail(h, GBS_ERR_INVALID, "free weights are required");
  const int m = n_dep + n_free;
  std::vector<int> steps(m);
  for (int k = 0; k < m; ++k) {
    const int N = k < n_dep ? steps_dep[k] : steps_free[k - n_dep];
    if (N < 2 || N > GBS_MAX_STEPS || N % 2) return fail(h, GBS_ERR_INVALID, "step count %d must be even in [2, %d]", N, GBS_MAX_STEPS);
    for (int l = 0; l < k; ++l)
      if (steps[l] == N) return fail(h, GBS_ERR_INVALID, "step count %d repeated", N);
    steps[k] = N;
  }
  Slot s;
  s.order = order_p;
  s.m = m;
  for (int k = 0; k < m; ++k) s.steps[k] = steps[k];
  char msg[200];
  gbs_status wst;
  if (c_full) {
    for (int k = 0; k < m; ++k) {
      if (!std::isfinite(c_full[k])) return fail(h, GBS_ERR_INVALID, "weight %d is not finite", k);
      s.c[k] = c_full[k];
    }
    wst = check_order_constraints(order_p, m, s.steps, s.c, msg, sizeof msg);
  } else {
    // c_dep from c_free (Sec. 3.7) in dd, then the order constraints with the rounded weights
    wst = scheme_weights(order_p, n_dep, n_free, s.steps, c_free, s.c, msg, sizeof msg);
  }
  if (wst != GBS_OK) return fail(h, wst, "%s", msg);
  s.isb = scan_isb(s);
  s.set = true;
  h->slots[slot] = s;
  if (h->adjoint) {
    int nmax = 0;
    for (int k = 0; k < m; ++k) nmax = std::max(nmax, steps[k]);
    if (nmax > h->levels_steps) {
      CK(h, cudaStreamSynchronize(h->stream));
      if (h->levels) cudaFree(h->levels);
      h->levels = nullptr;
      h->levels_steps = 0;
      gbs_status st = dalloc(h, &h->levels, (size_t)(nmax + 2) * h->state_elems * h->esz);
      if (st != GBS_OK) return st;
      h->levels_steps = nmax;
    }
  }
  return upload_slots(h);
}

gbs_status gbs_get_weights(gbs_handle h, int slot, int* m, int* steps, double* c, double* isb) {
  if (!h) return fail(nullptr, GBS_ERR_INVALID, "handle is NULL");
  if (slot < 0 || slot >= GBS_MAX_SLOTS) return fail(h, GBS_ERR_INVALID, "slot %d out of range", slot);
  const Slot& s = h->slots[slot];
  if (!s.set) return fail(h, GBS_ERR_STATE, "slot %d has no weights", slot);
  if (m) *m = s.m;
  for (int k = 0; k < s.m; ++k) {
    if (steps) steps[k] = s.steps[k];
    if (c) c[k] = s.c[k];
  }
  if (isb) *isb = s.isb;
  return GBS_OK;
}

gbs_status gbs_assign_slots(gbs_handle h, const int* slot_per_problem) {
  if (!h) return fail(nullptr, GBS_ERR_INVALID, "handle is NULL");
  if (!slot_per_problem) return fail(h, GBS_ERR_INVALID, "slot array is NULL");
  for (int p = 0; p < h->batch; ++p) {
    const int s = slot_per_problem[p];
    if (s < 0 || s >= GBS_MAX_SLOTS) return fail(h, GBS_ERR_INVALID, "problem %d: slot %d out of range", p, s);
    if (!h->slots[s].set) return fail(h, GBS_ERR_STATE, "problem %d: slot %d has no weights", p, s);
  }
  h->slot_of.assign(slot_per_problem, slot_per_problem + h->batch);
  return upload_slots(h);
}

gbs_status gbs_stability_limit(gbs_handle h, double* H_max) {
  if (!h) return fail(nullptr, GBS_ERR_INVALID, "handle is NULL");
  if (!H_max) return fail(h, GBS_ERR_INVALID, "H_max is NULL");
  const double smax = h->system == GBS_ONEWAY_SPECTRAL ? 0.0 : symbol_max(h->R);
  for (int p = 0; p < h->batch; ++p) {
    const Slot& s = h->slots[h->slot_of[p]];
    if (!s.set) return fail(h, GBS_ERR_STATE, "problem %d: slot %d has no weights", p, h->slot_of[p]);
    if (h->system == GBS_ONEWAY_SPECTRAL) {   // |i k| <= pi / dx on the grid (Sec. 4)
      H_max[p] = s.isb / (M_PI * h->probs[p].inv_dx[0]);
      continue;
    }
    double q = 0;
    for (int d = 0; d < h->ndim; ++d) q += (smax * h->probs[p].inv_dx[d]) * (smax * h->probs[p].inv_dx[d]);
    const double rho_hat = h->cmax[p] * std::sqrt(q);
    H_max[p] = s.isb / rho_hat;
  }
  return GBS_OK;
}

gbs_status gbs_step_batch(gbs_handle h, const void* y_in, void* y_out, const double* H, int n_macro) {
  if (!h) return fail(nullptr, GBS_ERR_INVALID, "handle is NULL");
  if (!H) return fail(h, GBS_ERR_INVALID, "H is NULL");
  if (n_macro < 0) return fail(h, GBS_ERR_INVALID, "n_macro must be >= 0");
  if (!y_in || !y_out) return fail(h, GBS_ERR_INVALID, "state pointers must not be NULL");
  const size_t bytes = (size_t)h->state_elems * h->esz;
  const char* a = static_cast<const char*>(y_in);
  const char* b = static_cast<const char*>(y_out);
  if (a != b && a < b + bytes && b < a + bytes) return fail(h, GBS_ERR_INVALID, "y_in and y_out overlap partially");
  StepPlan p;
  gbs_status st = build_plan(h, &p);
  if (st != GBS_OK) return st;
  st = set_H(h, H);
  if (st != GBS_OK) return st;
  if (h->opt_check_stability) {
    std::vector<double> hm(h->batch);
    if ((st = gbs_stability_limit(h, hm.data())) != GBS_OK) return st;
    for (int q = 0; q < h->batch; ++q)
      if (H[q] > hm[q]) return fail(h, GBS_ERR_UNSTABLE, "problem %d: H = %g exceeds the stability limit %g", q, H[q], hm[q]);
  }
  if (n_macro == 0) {
    if (a != b) CK(h, cudaMemcpyAsync(y_out, y_in, bytes, cudaMemcpyDeviceToDevice, h->stream));
    return GBS_OK;
  }
  if (h->fused_mask != ~0u) {   // a partial step planned the time-blocked kernel for fewer sequences
    h->fused_mask = ~0u;
    if ((st = prepare_fused(h)) != GBS_OK) return st;
  }
  for (int it = 0; it < n_macro; ++it) {
    st = run_macro(h, p, it == 0 ? y_in : y_out, y_out);
    if (st != GBS_OK) return st;
  }
  return GBS_OK;
}

gbs_status gbs_step(gbs_handle h, const void* y_in, void* y_out, double H, int n_macro) {
  if (!h) return fail(nullptr, GBS_ERR_INVALID, "handle is NULL");
  std::vector<double> Hs(h->batch, H);
  return gbs_step_batch(h, y_in, y_out, Hs.data(), n_macro);
}

gbs_status gbs_step_partial(gbs_handle h, const void* y_in, double* partial, double H, uint32_t seq_mask) {
  if (!h) return fail(nullptr, GBS_ERR_INVALID, "handle is NULL");
  if (!y_in || !partial) return fail(h, GBS_ERR_INVALID, "state pointers must not be NULL");
  if (h->system == GBS_ONEWAY_SPECTRAL) return fail(h, GBS_ERR_INVALID, "partial steps need a finite-difference system");
  if ((seq_mask & ((1u << GBS_MAX_SEQ) - 1u)) == 0) return fail(h, GBS_ERR_INVALID, "the sequence mask selects no sequence");
  StepPlan p;
  gbs_status st = build_plan(h, &p);
  if (st != GBS_OK) return st;
  std::vector<double> Hs(h->batch, H);
  if ((st = set_H(h, Hs.data())) != GBS_OK) return st;
  // problems whose slot has none of the selected sequences contribute zero
  CK(h, cudaMemsetAsync(partial, 0, sizeof(double) * (size_t)h->state_elems, h->stream));
  const bool fused = use_fused(h, p) && !h->ds;
  if (fused && h->fw_ready && h->fused_mask != seq_mask) {   // plan the time-blocked kernel for these sequences
    h->fused_mask = seq_mask;
    if ((st = prepare_fused(h)) != GBS_OK) return st;
  }
  p.seq_mask = seq_mask;
  p.partial = 1;
  p.acc = partial;
  const int n = fused && h->fw_ready    ? fused_partial_step(h->fw, p, y_in, partial, h->stream, h->d_err)
                : fused && h->tb3_ready ? tb3_macro_step(h->tb3, p, y_in, const_cast<void*>(y_in), h->stream)
                                        : plain_step(h, p, y_in, const_cast<void*>(y_in), h->stream);
  if (n < 0) return fail(h, GBS_ERR_CUDA, "kernel launch failed: %s", cudaGetErrorString(cudaGetLastError()));
  h->launches += n;
  return GBS_OK;
}

gbs_status gbs_combine_partial(gbs_handle h, const void* y_in, const double* total, void* y_out) {
  if (!h) return fail(nullptr, GBS_ERR_INVALID, "handle is NULL");
  if (!y_in || !total || !y_out) return fail(h, GBS_ERR_INVALID, "pointers must not be NULL");
  if (h->system == GBS_ONEWAY_SPECTRAL) return fail(h, GBS_ERR_INVALID, "partial steps need a finite-difference system");
  StepPlan p;
  gbs_status st = build_plan(h, &p);
  if (st != GBS_OK) return st;
  if (finish_partial(p, y_in, total, y_out, h->stream) < 0)
    return fail(h, GBS_ERR_CUDA, "kernel launch failed: %s", cudaGetErrorString(cudaGetLastError()));
  h->launches += 1;
  return GBS_OK;
}

gbs_status gbs_step_host(gbs_handle h, const void* y_in_host, void* y_out_host, double H, int n_macro) {
  if (!h) return fail(nullptr, GBS_ERR_INVALID, "handle is NULL");
  if (!y_in_host || !y_out_host) return fail(h, GBS_ERR_INVALID, "host buffers must not be NULL");
  const size_t bytes = (size_t)h->state_elems * h->esz;
  CK(h, cudaMemcpyAsync(h->stage, y_in_host, bytes, cudaMemcpyHostToDevice, h->stream));
  gbs_status st = gbs_step(h, h->stage, h->stage, H, n_macro);
  if (st != GBS_OK) return st;
  CK(h, cudaMemcpyAsync(y_out_host, h->stage, bytes, cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return GBS_OK;
}

gbs_status gbs_step_host_stream(gbs_handle h, const void* const* y_in_host, void* const* y_out_host, int count,
                                double H, int n_macro) {
  if (!h) return fail(nullptr, GBS_ERR_INVALID, "handle is NULL");
  if (count < 0 || (count > 0 && (!y_in_host || !y_out_host)))
    return fail(h, GBS_ERR_INVALID, "bad host buffer arrays");
  for (int i = 0; i < count; ++i)
    if (!y_in_host[i] || !y_out_host[i]) return fail(h, GBS_ERR_INVALID, "host buffer %d is NULL", i);
  const size_t bytes = (size_t)h->state_elems * h->esz;
  void* buf[2] = {h->stage, h->stage2};
  cudaStream_t hs = h->copy_stream, ds = h->d2h_stream;
  // input i goes to buf[i % 2].  Host-to-device copies run on hs, device-to-host copies on ds
  // (separate copy engines), the macro-steps on the handle's stream: step i waits for H2D(i),
  // D2H(i) waits for step i, and H2D(i + 1) into the other buffer waits for D2H(i - 1), the
  // buffer's previous reader (which itself waited for step i - 1).  So H2D(i + 1) and D2H(i - 1)
  // overlap step i.  Both copy streams first wait for the handle's stream's earlier work.
  CK(h, cudaEventRecord(h->ev_out[0], h->stream));
  CK(h, cudaStreamWaitEvent(hs, h->ev_out[0], 0));
  CK(h, cudaStreamWaitEvent(ds, h->ev_out[0], 0));
  if (count > 0) {
    CK(h, cudaMemcpyAsync(buf[0], y_in_host[0], bytes, cudaMemcpyHostToDevice, hs));
    CK(h, cudaEventRecord(h->ev_in[0], hs));
  }
  for (int i = 0; i < count; ++i) {
    const int b = i & 1;
    CK(h, cudaStreamWaitEvent(h->stream, h->ev_in[b], 0));
    gbs_status st = gbs_step(h, buf[b], buf[b], H, n_macro);
    if (st != GBS_OK) {
      cudaStreamSynchronize(hs);
      cudaStreamSynchronize(ds);
      return st;
    }
    CK(h, cudaEventRecord(h->ev_out[b], h->stream));
    if (i + 1 < count) {
      if (i >= 1) CK(h, cudaStreamWaitEvent(hs, h->ev_d2h[b ^ 1], 0));
      CK(h, cudaMemcpyAsync(buf[b ^ 1], y_in_host[i + 1], bytes, cudaMemcpyHostToDevice, hs));
      CK(h, cudaEventRecord(h->ev_in[b ^ 1], hs));
    }
    CK(h, cudaStreamWaitEvent(ds, h->ev_out[b], 0));
    CK(h, cudaMemcpyAsync(y_out_host[i], buf[b], bytes, cudaMemcpyDeviceToHost, ds));
    CK(h, cudaEventRecord(h->ev_d2h[b], ds));
  }
  CK(h, cudaStreamSynchronize(hs));
  CK(h, cudaStreamSynchronize(ds));
  CK(h, cudaStreamSynchronize(h->stream));
  return GBS_OK;
}

gbs_status gbs_adjoint_step(gbs_handle h, const void* y_in, const void* lam_out, void* lam_in, double* grad_kappa,
                            double H, const int64_t* rcv_idx, int n_rcv, const void* rcv_resid) {
  if (!h) return fail(nullptr, GBS_ERR_INVALID, "handle is NULL");
  if (!h->adjoint) return fail(h, GBS_ERR_STATE, "handle was created without enable_adjoint");
  if (!y_in || !lam_out || !lam_in || !grad_kappa) return fail(h, GBS_ERR_INVALID, "pointers must not be NULL");
  if (n_rcv < 0 || (n_rcv > 0 && (!rcv_idx || !rcv_resid))) return fail(h, GBS_ERR_INVALID, "bad receiver arguments");
  if (n_rcv > 0 && h->batch != 1) return fail(h, GBS_ERR_INVALID, "receivers need batch == 1");
  AdjPlan a;
  gbs_status st = build_plan(h, &a.fw);
  if (st != GBS_OK) return st;
  for (int k = 0; k < a.fw.max_m; ++k)
    if (a.fw.max_steps_k[k] > h->levels_steps) return fail(h, GBS_ERR_STATE, "adjoint level store too small");
  std::vector<double> Hs(h->batch, H);
  if ((st = set_H(h, Hs.data())) != GBS_OK) return st;
  a.levels = h->levels;
  a.mu0 = h->mu0;
  a.mu1 = h->mu1;
  a.shared = h->mu_shared;
  a.gpair = h->gpair;
  a.max_steps = h->levels_steps;
  a.rcv_pts = h->probs[0].pts;
  a.err = h->d_err;
  // FP64 states in FP32 pairs: the adjoint in pair arithmetic, with the second staging state
  // (idle outside gbs_step_host_stream) as the pair copy of lam_out
  const int n = h->ds ? plain_adjoint_step_pairs(a, h->stage2, y_in, lam_out, lam_in, grad_kappa, rcv_idx, n_rcv,
                                                 rcv_resid, h->stream)
                      : plain_adjoint_step(a, y_in, lam_out, lam_in, grad_kappa, rcv_idx, n_rcv, rcv_resid, h->stream);
  if (n < 0) return fail(h, GBS_ERR_CUDA, "adjoint launch failed: %s", cudaGetErrorString(cudaGetLastError()));
  h->launches += n;
  return GBS_OK;
}

gbs_status gbs_misfit(gbs_handle h, const void* y, const int64_t* rcv_idx, int n_rcv, const void* data, void* resid,
                      double* J) {
  if (!h) return fail(nullptr, GBS_ERR_INVALID, "handle is NULL");
  if (!y || !rcv_idx || !data || n_rcv < 0) return fail(h, GBS_ERR_INVALID, "bad misfit arguments");
  if (n_rcv == 0) return GBS_OK;
  if (misfit(h->f64, y, rcv_idx, n_rcv, data, resid, J, h->probs[0].pts, h->d_err, h->stream) < 0)
    return fail(h, GBS_ERR_CUDA, "misfit launch failed: %s", cudaGetErrorString(cudaGetLastError()));
  h->launches += 1;
  return GBS_OK;
}

gbs_status gbs_inject(gbs_handle h, void* lam, const int64_t* rcv_idx, int n_rcv, const void* values) {
  if (!h) return fail(nullptr, GBS_ERR_INVALID, "handle is NULL");
  if (!lam || n_rcv < 0 || (n_rcv > 0 && (!rcv_idx || !values))) return fail(h, GBS_ERR_INVALID, "bad inject arguments");
  const int n = inject(h->f64, lam, rcv_idx, n_rcv, values, h->probs[0].pts, h->d_err, h->stream);
  if (n < 0) return fail(h, GBS_ERR_CUDA, "inject launch failed: %s", cudaGetErrorString(cudaGetLastError()));
  h->launches += n;
  return GBS_OK;
}

gbs_status gbs_norms(gbs_handle h, const void* a, const void* b, double* out) {
  if (!h) return fail(nullptr, GBS_ERR_INVALID, "handle is NULL");
  if (!a || !out) return fail(h, GBS_ERR_INVALID, "bad norms arguments");
  const int n = norms(h->f64, a, b, h->state_elems, h->d_red, h->d_red + 4 * kNormBlocks, h->stream);
  if (n < 0) return fail(h, GBS_ERR_CUDA, "norms launch failed: %s", cudaGetErrorString(cudaGetLastError()));
  h->launches += n;
  CK(h, cudaMemcpyAsync(out, h->d_red + 4 * kNormBlocks, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  return GBS_OK;
}

gbs_status gbs_set_option(gbs_handle h, const char* name, int64_t value) {
  if (!h) return fail(nullptr, GBS_ERR_INVALID, "handle is NULL");
  if (!name) return fail(h, GBS_ERR_INVALID, "option name is NULL");
  if (!std::strcmp(name, "kernel")) {
    if (value < GBS_KERNEL_AUTO || value > GBS_KERNEL_FUSED) return fail(h, GBS_ERR_INVALID, "bad kernel option");
    if (value == GBS_KERNEL_FUSED) {
      StepPlan p;
      gbs_status st = build_plan(h, &p);
      if (st != GBS_OK) return st;
      SlotDev sd[GBS_MAX_SLOTS];
      std::memset(sd, 0, sizeof sd);
      for (int i = 0; i < GBS_MAX_SLOTS; ++i) {
        sd[i].m = h->slots[i].m;
        for (int k = 0; k < h->slots[i].m; ++k) sd[i].steps[k] = h->slots[i].steps[k];
      }
      if (!fused_supported(p, h->probs.data()) && !tb3_supported(p, h->probs.data(), sd, GBS_MAX_SLOTS))
        return fail(h, GBS_ERR_INVALID, "the time-blocked kernel does not support this problem");
    }
    h->opt_kernel = (int)value;
    gbs_status st = prepare_fused(h);
    if (st != GBS_OK) return st;
  } else if (!std::strcmp(name, "graph")) {
    h->opt_graph = value != 0;
  } else if (!std::strcmp(name, "check_stability")) {
    h->opt_check_stability = value != 0;
  } else if (!std::strcmp(name, "hseg")) {
    if (value < 16 || value > 65536) return fail(h, GBS_ERR_INVALID, "hseg must be in [16, 65536]");
    h->opt_hseg = (int)value;
    gbs_status st = prepare_fused(h);
    if (st != GBS_OK) return st;
  } else if (!std::strcmp(name, "seqgroup")) {
    if (value < -1 || value > GBS_MAX_SEQ) return fail(h, GBS_ERR_INVALID, "seqgroup must be in [-1, %d]", GBS_MAX_SEQ);
    h->opt_seqgroup = (int)value;
  } else if (!std::strcmp(name, "seqfuse")) {
    if (value != 0 && value != 1) return fail(h, GBS_ERR_INVALID, "seqfuse must be 0 or 1");
    h->opt_seqfuse = (int)value;
    gbs_status st = prepare_fused(h);
    if (st != GBS_OK) return st;
  } else if (!std::strcmp(name, "zseg")) {
    if (value < 1 || value > 65536) return fail(h, GBS_ERR_INVALID, "zseg must be in [1, 65536]");
    h->opt_zseg = (int)value;
    gbs_status st = prepare_fused(h);
    if (st != GBS_OK) return st;
  } else if (!std::strcmp(name, "tmax")) {
    if (value != 0 && (value < 2 || value > fused_max_levels() || value % 2))
      return fail(h, GBS_ERR_INVALID, "tmax must be 0 or even in [2, %d]", fused_max_levels());
    h->opt_tmax = (int)value;
    gbs_status st = prepare_fused(h);
    if (st != GBS_OK) return st;
  } else if (!std::strcmp(name, "schedule")) {
    if (value != 0 && value != 1) return fail(h, GBS_ERR_INVALID, "schedule must be 0 or 1");
    h->opt_schedule = (int)value;
    gbs_status st = prepare_fused(h);
    if (st != GBS_OK) return st;
  } else if (!std::strcmp(name, "spin_limit") || !std::strcmp(name, "inject_unsatisfiable_wait")) {
    if (!std::strcmp(name, "spin_limit")) {
      if (value < 1) return fail(h, GBS_ERR_INVALID, "spin_limit must be >= 1");
      h->opt_spin_limit = value;
    } else {
      h->opt_inject_wait = value != 0;
    }
    fused_set_test_hooks(h->fw, h->opt_spin_limit, h->opt_inject_wait);
    gbs_status st = prepare_fused(h);
    if (st != GBS_OK) return st;
  } else if (!std::strcmp(name, "tma")) {
    if (value < -1 || value > 1) return fail(h, GBS_ERR_INVALID, "tma must be -1, 0 or 1");
    h->opt_tma = (int)value;
  } else if (!std::strcmp(name, "combine")) {
    if (value != 0 && value != 1) return fail(h, GBS_ERR_INVALID, "combine must be 0 (FP64) or 1 (FP32 pairs)");
    h->opt_combine = (int)value;
    fused_set_combine(h->fw, value == 0);
  } else if (!std::strcmp(name, "time_kernels")) {
    if (value && h->tev.empty()) {
      const int pairs = 8192;
      h->tev.resize(2 * pairs);
      h->tev_bytes.assign(pairs, 0.0);
      for (auto& e : h->tev) CK(h, cudaEventCreate(&e));
    }
    h->opt_time_kernels = value != 0;
    h->tev_used = 0;
  } else {
    return fail(h, GBS_ERR_INVALID, "unknown option '%s'", name);
  }
  ++h->sched_version;
  return GBS_OK;
}

gbs_status gbs_get_option(gbs_handle h, const char* name, int64_t* value) {
  if (!h) return fail(nullptr, GBS_ERR_INVALID, "handle is NULL");
  if (!name || !value) return fail(h, GBS_ERR_INVALID, "bad arguments");
  if (!std::strcmp(name, "kernel")) *value = h->opt_kernel;
  else if (!std::strcmp(name, "graph")) *value = h->opt_graph;
  else if (!std::strcmp(name, "check_stability")) *value = h->opt_check_stability;
  else if (!std::strcmp(name, "time_kernels")) *value = h->opt_time_kernels;
  else if (!std::strcmp(name, "hseg")) *value = h->opt_hseg;
  else if (!std::strcmp(name, "zseg")) *value = h->opt_zseg;
  else if (!std::strcmp(name, "seqfuse")) *value = h->ms_ready ? 1 : 0;
  else if (!std::strcmp(name, "seqgroup")) *value = h->opt_seqgroup >= 0 ? h->opt_seqgroup : h->ndim == 3 ? kSeqGroup3D : 0;
  else if (!std::strcmp(name, "tmax")) *value = h->opt_tmax ? h->opt_tmax : fused_max_levels();
  else if (!std::strcmp(name, "schedule")) *value = h->opt_schedule;
  else if (!std::strcmp(name, "tma")) *value = tma_in_use(h) ? 1 : 0;
  else if (!std::strcmp(name, "spin_limit")) *value = h->opt_spin_limit;
  else if (!std::strcmp(name, "inject_unsatisfiable_wait")) *value = h->opt_inject_wait;
  else if (!std::strcmp(name, "combine")) *value = h->opt_combine;
  else if (!std::strcmp(name, "kernel_in_use")) {
    StepPlan p;
    gbs_status st = build_plan(h, &p);
    if (st != GBS_OK) return st;
    *value = use_fused(h, p) ? GBS_KERNEL_FUSED : GBS_KERNEL_PLAIN;
  } else return fail(h, GBS_ERR_INVALID, "unknown option '%s'", name);
  return GBS_OK;
}

gbs_status gbs_kernel_time(gbs_handle h, int64_t* launches, double* total_ms, double* bytes) {
  if (!h) return fail(nullptr, GBS_ERR_INVALID, "handle is NULL");
  if (!launches || !total_ms) return fail(h, GBS_ERR_INVALID, "output pointers must not be NULL");
  CK(h, cudaStreamSynchronize(h->stream));
  double ms = 0, by = 0;
  for (int u = 0; u < h->tev_used; ++u) {
    float t = 0;
    CK(h, cudaEventElapsedTime(&t, h->tev[2 * u], h->tev[2 * u + 1]));
    ms += t;
    by += h->tev_bytes[u];
  }
  *launches = h->tev_used;
  *total_ms = ms;
  if (bytes) *bytes = by;
  h->tev_used = 0;
  return GBS_OK;
}

gbs_status gbs_sync(gbs_handle h) {
  if (!h) return fail(nullptr, GBS_ERR_INVALID, "handle is NULL");
  CK(h, cudaStreamSynchronize(h->stream));
  int flag = 0;
  CK(h, cudaMemcpy(&flag, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    cudaMemset(h->d_err, 0, sizeof(int));
    if (flag == GBS_ERR_TIMEOUT) return fail(h, GBS_ERR_TIMEOUT, "a device-side wait timed out");
    return fail(h, (gbs_status)flag, "device-side error %d", flag);
  }
  return GBS_OK;
}

gbs_status gbs_destroy(gbs_handle h) {
  if (!h) return GBS_OK;
  cudaStreamSynchronize(h->stream);
  free_all(h);
  delete h;
  return GBS_OK;
}

const char* gbs_last_error(gbs_handle h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int64_t gbs_kernel_launches(gbs_handle h) { return h ? h->launches : 0; }

}  // extern "C"
