// gbs_step_noalloc: advance a problem by extrapolated GBS macro-steps without
// allocating any memory.
//
// Who needs this: code that must not (or cannot) call cudaMalloc -- for example
// a host application whose GPU memory is entirely handed out by its own
// allocator or memory pool, a plug-in loaded into such a process, or a caller
// that is not allowed to grow the device heap at the point where it steps.
// gbs_create() allocates its workspace with cudaMalloc, so those callers cannot
// use a handle.  This entry point instead keeps its scratch (leap-frog levels,
// shared first right-hand side, FP64 combine accumulator, 1/rho and the small
// problem tables) in one fixed array compiled into the library.
//
// The array below is a file-scope __device__ variable: every GPU on which the
// library is loaded reserves kNoAllocScratchBytes for it until the process
// exits.  Host code cannot use the name of the array as a device address (in
// host code it names a host-side shadow), so the device address is looked up
// with cudaGetSymbolAddress once per device, on the first call made while that
// device is current.  The small problem tables are copied into the array from
// pageable host memory, so every call waits until the work queued earlier on
// its stream has finished before it returns, and no call may be made while
// its stream is being captured (such a call is refused with GBS_ERR_STATE
// before anything is enqueued).  All calls on a device share the one array:
// calls whose GPU work overlaps in time (different streams, or different host
// threads) race on it.  The array keeps whatever the previous call left in it;
// nothing in it needs to start at zero because every buffer is fully written
// before it is read.  kappa and rho are used as given: unlike gbs_create, this
// entry point does not check them for non-positive or non-finite values.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "gbs_internal.h"
#include "gbs_weights.h"

namespace {

constexpr size_t kNoAllocScratchBytes = GBS_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};
thread_local char g_noalloc_err[256] = {0};

gbs_status noalloc_fail(gbs_status st, const char* msg) {
  std::strncpy(g_noalloc_err, msg, sizeof g_noalloc_err - 1);
  return st;
}

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

// Device address of the scratch array on the current device (looked up once per device).
gbs_status scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return noalloc_fail(GBS_ERR_CUDA, "gbs_step_noalloc: no usable current CUDA device");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return noalloc_fail(GBS_ERR_CUDA, "gbs_step_noalloc: cudaGetSymbolAddress of the scratch array failed");
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return GBS_OK;
}

}  // namespace

extern "C" const char* gbs_noalloc_last_error(void) { return g_noalloc_err; }

extern "C" gbs_status gbs_step_noalloc(const gbs_problem* pb, const void* kappa, const void* rho, int order_p,
                                       int n_dep, const int* steps_dep, int n_free, const int* steps_free,
                                       const double* c_free, const void* y_in, void* y_out, double H, int n_macro,
                                       void* cuda_stream) {
  using namespace gbs;
  g_noalloc_err[0] = 0;
  // ---- problem description (no heap use anywhere below) ----
  if (!pb) return noalloc_fail(GBS_ERR_INVALID, "problem description is NULL");
  if (pb->system != GBS_WAVE1D && pb->system != GBS_ACOUSTIC)
    return noalloc_fail(GBS_ERR_INVALID, "system must be GBS_WAVE1D or GBS_ACOUSTIC");
  if (pb->ndim < 1 || pb->ndim > 3 || (pb->system == GBS_WAVE1D && pb->ndim != 1))
    return noalloc_fail(GBS_ERR_INVALID, "bad ndim");
  if (pb->fd_order != 4 && pb->fd_order != 6) return noalloc_fail(GBS_ERR_INVALID, "fd_order must be 4 or 6");
  if (pb->precision != GBS_F32_STATE_F64_COMBINE && pb->precision != GBS_F64)
    return noalloc_fail(GBS_ERR_INVALID, "unknown precision");
  if (pb->enable_adjoint) return noalloc_fail(GBS_ERR_INVALID, "gbs_step_noalloc has no adjoint");
  if (pb->batch < 1 || pb->batch > 256) return noalloc_fail(GBS_ERR_INVALID, "batch must be in [1, 256]");
  if (!pb->shape || !pb->dx) return noalloc_fail(GBS_ERR_INVALID, "shape and dx arrays are required");
  if ((pb->system == GBS_ACOUSTIC) != (kappa != nullptr && rho != nullptr))
    return noalloc_fail(GBS_ERR_INVALID, "acoustics needs kappa and rho; the 1D wave system takes none");
  if (!y_in || !y_out) return noalloc_fail(GBS_ERR_INVALID, "state pointers must not be NULL");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  {
    // the tables below are uploaded from pageable host memory, which a stream capture cannot
    // record: refuse before anything is enqueued, so the caller's capture stays valid
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
      cudaGetLastError();
      return noalloc_fail(GBS_ERR_CUDA, "gbs_step_noalloc: cudaStreamIsCapturing failed");
    }
    if (cs != cudaStreamCaptureStatusNone)
      return noalloc_fail(GBS_ERR_STATE, "gbs_step_noalloc must not be called while its stream is being captured");
  }
  for (const void* ptr : {kappa, rho, static_cast<const void*>(y_in), static_cast<const void*>(y_out)}) {
    if (!ptr) continue;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess ||
        (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
      cudaGetLastError();
      return noalloc_fail(GBS_ERR_INVALID, "kappa, rho, y_in and y_out must be device pointers");
    }
  }
  if (!(H > 0) || !std::isfinite(H) || n_macro < 0) return noalloc_fail(GBS_ERR_INVALID, "bad H or n_macro");
  const int F = pb->system == GBS_WAVE1D ? 2 : 1 + pb->ndim;
  const int R = pb->fd_order / 2;
  const size_t esz = pb->precision == GBS_F64 ? 8 : 4;
  // ---- scheme: dependent weights by Bjorck-Pereyra in double-double (Sec. 3.7) ----
  if (order_p < 2 || order_p % 2 || n_dep != order_p / 2 || n_free < 0 || n_dep + n_free > GBS_MAX_SEQ)
    return noalloc_fail(GBS_ERR_INVALID, "bad order or number of sequences");
  if (!steps_dep || (n_free > 0 && (!steps_free || !c_free))) return noalloc_fail(GBS_ERR_INVALID, "scheme arrays missing");
  const int m = n_dep + n_free;
  SlotDev slot;
  std::memset(&slot, 0, sizeof slot);
  slot.m = m;
  for (int k = 0; k < m; ++k) {
    const int N = k < n_dep ? steps_dep[k] : steps_free[k - n_dep];
    if (N < 2 || N > GBS_MAX_STEPS || N % 2) return noalloc_fail(GBS_ERR_INVALID, "step counts must be even in [2, 64]");
    for (int l = 0; l < k; ++l)
      if (slot.steps[l] == N) return noalloc_fail(GBS_ERR_INVALID, "step counts must be distinct");
    slot.steps[k] = N;
  }
  {
    // c_dep from c_free in double-double and the order constraints with the rounded weights,
    // exactly as gbs_set_weights does (Sec. 3.7)
    char msg[200];
    const gbs_status wst = scheme_weights(order_p, n_dep, n_free, slot.steps, c_free, slot.c, msg, sizeof msg);
    if (wst != GBS_OK) return noalloc_fail(wst, msg);
    split_weights(slot);
  }
  // ---- layout inside the scratch array ----
  ProbDev probs[256];
  int64_t soff = 0, moff = 0, blk = 0;
  for (int p = 0; p < pb->batch; ++p) {
    ProbDev& d = probs[p];
    std::memset(&d, 0, sizeof d);
    for (int k = 0; k < 3; ++k) {
      const int64_t n = pb->shape[3 * p + k];
      if (k < pb->ndim) {
        if (n < R || n > (int64_t(1) << 30)) return noalloc_fail(GBS_ERR_INVALID, "grid size out of range");
        if (!(pb->dx[3 * p + k] > 0) || !std::isfinite(pb->dx[3 * p + k]))
          return noalloc_fail(GBS_ERR_INVALID, "dx must be finite and > 0");
        d.inv_dx[k] = 1.0 / pb->dx[3 * p + k];
      } else if (n != 1) {
        return noalloc_fail(GBS_ERR_INVALID, "unused dimensions must have size 1");
      }
      d.n[k] = (int)n;
    }
    fill_fp32_consts(d, pb->ndim, R);
    d.pts = (int64_t)d.n[0] * d.n[1] * d.n[2];
    if (d.pts >= (int64_t(1) << 31)) return noalloc_fail(GBS_ERR_INVALID, "a problem has 2^31 or more points");
    d.slot = 0;
    d.state_off = soff;
    d.media_off = moff;
    d.blk_begin = blk;
    soff += F * d.pts;
    moff += d.pts;
    blk += (d.pts + kPlainBlock - 1) / kPlainBlock;
  }
  const int64_t tiles = assign_tiles(probs, pb->batch, pb->ndim);
  const size_t o_probs = 0;
  const size_t o_slot = align256(o_probs + sizeof(ProbDev) * pb->batch);
  const size_t o_H = align256(o_slot + sizeof(SlotDev));
  const size_t o_hk = align256(o_H + sizeof(double) * pb->batch);
  const size_t o_hkf = align256(o_hk + sizeof(double) * pb->batch * GBS_MAX_SEQ);
  const size_t o_hkq = align256(o_hkf + sizeof(float2) * pb->batch * GBS_MAX_SEQ);
  const size_t o_b = align256(o_hkq + sizeof(float4) * pb->batch * GBS_MAX_SEQ);
  const size_t o_f0 = align256(o_b + (pb->system == GBS_ACOUSTIC ? moff * esz : 0));
  const size_t o_L0 = align256(o_f0 + soff * esz);
  const size_t o_L1 = align256(o_L0 + soff * esz);
  const size_t o_acc = align256(o_L1 + soff * esz);
  const size_t need = o_acc + soff * sizeof(double);
  if (need > kNoAllocScratchBytes) {
    char msg[200];
    std::snprintf(msg, sizeof msg, "problem needs %zu bytes of scratch; gbs_step_noalloc is limited to %zu bytes",
                  need, kNoAllocScratchBytes);
    return noalloc_fail(GBS_ERR_INVALID, msg);
  }
  const size_t bytes = (size_t)soff * esz;
  const char* a = static_cast<const char*>(y_in);
  const char* b = static_cast<const char*>(y_out);
  if (a != b && a < b + bytes && b < a + bytes) return noalloc_fail(GBS_ERR_INVALID, "y_in and y_out overlap partially");
  void* base = nullptr;
  gbs_status st = scratch_address(&base);
  if (st != GBS_OK) return st;
  char* sc = static_cast<char*>(base);
  // host staging of the per-problem step tables: automatic arrays (about 130 KB of stack)
  double Hs[256];
  double hk[256 * GBS_MAX_SEQ];
  float2 hkf[256 * GBS_MAX_SEQ];
  float4 hkq[256 * GBS_MAX_SEQ];
  for (int p = 0; p < pb->batch; ++p) {
    Hs[p] = H;
    for (int k = 0; k < GBS_MAX_SEQ; ++k) {
      hk[p * GBS_MAX_SEQ + k] = k < m ? H / slot.steps[k] : 0.0;
      hkf[p * GBS_MAX_SEQ + k] = make_float2((float)hk[p * GBS_MAX_SEQ + k], (float)(2.0 * hk[p * GBS_MAX_SEQ + k]));
      hkq[p * GBS_MAX_SEQ + k] = fp32_step_consts(probs[p], hk[p * GBS_MAX_SEQ + k], R);
    }
  }
  // pageable sources: each copy returns once its data are staged, so the stack arrays may go
  if (cudaMemcpyAsync(sc + o_probs, probs, sizeof(ProbDev) * pb->batch, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(sc + o_slot, &slot, sizeof(SlotDev), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(sc + o_H, Hs, sizeof(double) * pb->batch, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(sc + o_hk, hk, sizeof(double) * pb->batch * GBS_MAX_SEQ, cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(sc + o_hkf, hkf, sizeof(float2) * pb->batch * GBS_MAX_SEQ, cudaMemcpyHostToDevice, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(sc + o_hkq, hkq, sizeof(float4) * pb->batch * GBS_MAX_SEQ, cudaMemcpyHostToDevice, s) !=
          cudaSuccess) {
    cudaGetLastError();
    return noalloc_fail(GBS_ERR_CUDA, "gbs_step_noalloc: table upload failed");
  }
  if (pb->system == GBS_ACOUSTIC && prep_media(pb->precision == GBS_F64, rho, sc + o_b, moff, s) < 0)
    return noalloc_fail(GBS_ERR_CUDA, "gbs_step_noalloc: media kernel launch failed");
  if (n_macro == 0) {
    if (a != b && cudaMemcpyAsync(y_out, y_in, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return noalloc_fail(GBS_ERR_CUDA, "gbs_step_noalloc: copy failed");
    return GBS_OK;
  }
  StepPlan p;
  std::memset(&p, 0, sizeof p);
  p.system = pb->system;
  p.ndim = pb->ndim;
  p.R = R;
  p.f64 = pb->precision == GBS_F64;
  p.F = F;
  p.batch = pb->batch;
  p.probs = reinterpret_cast<const ProbDev*>(sc + o_probs);
  p.slots = reinterpret_cast<const SlotDev*>(sc + o_slot);
  p.H = reinterpret_cast<const double*>(sc + o_H);
  p.hk = reinterpret_cast<const double*>(sc + o_hk);
  p.hkf = reinterpret_cast<const float2*>(sc + o_hkf);
  p.hkq = reinterpret_cast<const float4*>(sc + o_hkq);
  p.total_blocks = blk;
  p.total_tiles = tiles;
  p.state_elems = soff;
  p.kappa = kappa;
  p.b = sc + o_b;
  p.f0 = sc + o_f0;
  p.L0 = sc + o_L0;
  p.L1 = sc + o_L1;
  p.acc = reinterpret_cast<double*>(sc + o_acc);
  p.max_m = m;
  p.seq_mask = ~0u;
  for (int k = 0; k < m; ++k) p.max_steps_k[k] = slot.steps[k];
  for (int it = 0; it < n_macro; ++it) {
    if (plain_macro_step(p, it == 0 ? y_in : y_out, y_out, s) < 0) {
      cudaGetLastError();
      return noalloc_fail(GBS_ERR_CUDA, "gbs_step_noalloc: kernel launch failed");
    }
  }
  return GBS_OK;
}
