// Media preparation and reductions: b = 1/rho, per-problem max wave speed,
// state norms and the receiver misfit.  Reductions accumulate in FP64 with
// warp shuffles, then shared memory, then a fixed-order second pass, so the
// results do not depend on scheduling.
#include <cuda_runtime.h>

#include <cmath>

#include "gbs_internal.h"
#include "gbs_stencil.cuh"

namespace gbs {
namespace {

template <typename T>
__global__ void k_recip(const T* __restrict__ rho, T* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = T(1) / rho[i];
}

// out[p] = max_i sqrt(kappa_i b_i) over problem p (atomicMax on the bit pattern of a
// non-negative double is order independent).
template <typename T>
__global__ void k_cmax(const T* __restrict__ kappa, const T* __restrict__ b, const ProbDev* probs,
                       double* out) {
  const ProbDev q = probs[blockIdx.y];
  double m = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < q.pts; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = sqrt((double)kappa[q.media_off + i] * (double)b[q.media_off + i]);
    m = fmax(m, v);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0)
    atomicMax(reinterpret_cast<unsigned long long*>(out + blockIdx.y), (unsigned long long)__double_as_longlong(m));
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

constexpr int kRedThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_norms_partial(const T* __restrict__ a, const T* __restrict__ b,
                                                               int64_t n, double* partial) {
  double sd = 0, sb = 0, mx = 0, nf = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double av = (double)a[i];
    const double bv = b ? (double)b[i] : 0.0;
    if (!isfinite(av)) {
      nf += 1;
      continue;
    }
    const double d = av - bv;
    sd += d * d;
    sb += bv * bv;
    mx = fmax(mx, fabs(d));
  }
  __shared__ double sh[4][kRedThreads / 32];
  sd = warp_sum(sd);
  sb = warp_sum(sb);
  mx = warp_max(mx);
  nf = warp_sum(nf);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sh[0][w] = sd;
    sh[1][w] = sb;
    sh[2][w] = mx;
    sh[3][w] = nf;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double r0 = 0, r1 = 0, r2 = 0, r3 = 0;
    for (int i = 0; i < kRedThreads / 32; ++i) {
      r0 += sh[0][i];
      r1 += sh[1][i];
      r2 = fmax(r2, sh[2][i]);
      r3 += sh[3][i];
    }
    partial[4 * blockIdx.x + 0] = r0;
    partial[4 * blockIdx.x + 1] = r1;
    partial[4 * blockIdx.x + 2] = r2;
    partial[4 * blockIdx.x + 3] = r3;
  }
}

__global__ void k_norms_final(const double* partial, int nb, double* out) {
  // one warp, fixed order
  double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  for (int i = threadIdx.x; i < nb; i += 32) {
    s0 += partial[4 * i + 0];
    s1 += partial[4 * i + 1];
    s2 = fmax(s2, partial[4 * i + 2]);
    s3 += partial[4 * i + 3];
  }
  s0 = warp_sum(s0);
  s1 = warp_sum(s1);
  s2 = warp_max(s2);
  s3 = warp_sum(s3);
  if (threadIdx.x == 0) {
    out[0] = s0;
    out[1] = s1;
    out[2] = s2;
    out[3] = s3;
  }
}

template <typename T>
__global__ void k_misfit(const T* __restrict__ y, const int64_t* __restrict__ idx, int n,
                         const T* __restrict__ data, T* __restrict__ resid, double* J, int64_t n_valid,
                         int* err) {
  __shared__ double sh[32];
  double s = 0;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const int64_t i = idx[r];
    if (i < 0 || i >= n_valid) {   // out-of-range receiver: latch an error, skip it
      atomicCAS(err, 0, (int)GBS_ERR_INVALID);
      if (resid) resid[r] = T(0);
      continue;
    }
    const T v = y[i] - data[r];
    if (resid) resid[r] = v;
    s += (double)v * (double)v;
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0 && J) {
    double t = 0;
    for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) t += sh[i];
    *J += 0.5 * t;
  }
}

}  // namespace

int prep_media(int f64, const void* rho, void* b, int64_t n, cudaStream_t s) {
  if (f64) k_recip<double><<<1024, 256, 0, s>>>(static_cast<const double*>(rho), static_cast<double*>(b), n);
  else k_recip<float><<<1024, 256, 0, s>>>(static_cast<const float*>(rho), static_cast<float*>(b), n);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int media_cmax(int f64, const void* kappa, const void* b, const ProbDev* probs, int batch, double* out,
               cudaStream_t s) {
  if (cudaMemsetAsync(out, 0, sizeof(double) * batch, s) != cudaSuccess) return -1;
  const dim3 grid(64, batch);
  if (f64) k_cmax<double><<<grid, 256, 0, s>>>(static_cast<const double*>(kappa), static_cast<const double*>(b), probs, out);
  else k_cmax<float><<<grid, 256, 0, s>>>(static_cast<const float*>(kappa), static_cast<const float*>(b), probs, out);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int norms(int f64, const void* a, const void* b, int64_t n, double* partial, double* out4, cudaStream_t s) {
  int64_t nb = (n + kRedThreads - 1) / kRedThreads;
  if (nb > kNormBlocks) nb = kNormBlocks;
  if (nb < 1) nb = 1;
  if (f64)
    k_norms_partial<double><<<(unsigned)nb, kRedThreads, 0, s>>>(static_cast<const double*>(a), static_cast<const double*>(b), n, partial);
  else
    k_norms_partial<float><<<(unsigned)nb, kRedThreads, 0, s>>>(static_cast<const float*>(a), static_cast<const float*>(b), n, partial);
  k_norms_final<<<1, 32, 0, s>>>(partial, (int)nb, out4);
  return cudaPeekAtLastError() == cudaSuccess ? 2 : -1;
}

int misfit(int f64, const void* y, const int64_t* idx, int n_rcv, const void* data, void* resid, double* J,
           int64_t n_valid, int* err, cudaStream_t s) {
  if (f64)
    k_misfit<double><<<1, 256, 0, s>>>(static_cast<const double*>(y), idx, n_rcv, static_cast<const double*>(data),
                                       static_cast<double*>(resid), J, n_valid, err);
  else
    k_misfit<float><<<1, 256, 0, s>>>(static_cast<const float*>(y), idx, n_rcv, static_cast<const float*>(data),
                                      static_cast<float*>(resid), J, n_valid, err);
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace gbs

// ---------------------------------------------------------------------------
// Self-test of the exact FP32 -> FP64 promotion used by the FP64 combines (promote, in
// gbs_stencil.cuh): its bits against the conversion instruction's for a range of float bit
// patterns.  Counters live in a small static device array (the call allocates nothing).
// ---------------------------------------------------------------------------
namespace gbs {
namespace {

// [0] inputs that are not NaN and whose doubles differ; [1] NaN inputs whose doubles differ in
// more than the quiet bit (bit 51); [2] NaN inputs whose doubles differ in the quiet bit alone
__device__ unsigned long long g_promote_mismatch[3];

__global__ void __launch_bounds__(256) k_selftest_promote(unsigned long long first, unsigned long long count) {
  unsigned long long bad = 0, badnan = 0, quiet = 0;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < count;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned b = (unsigned)(first + i);
    const float f = __uint_as_float(b);
    const unsigned long long x = (unsigned long long)__double_as_longlong(promote(f)) ^
                                 (unsigned long long)__double_as_longlong((double)f);
    if (x) {
      if ((b & 0x7fffffffu) <= 0x7f800000u) ++bad;
      else if (x == (1ull << 51)) ++quiet;
      else ++badnan;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    bad += __shfl_down_sync(0xffffffffu, bad, o);
    badnan += __shfl_down_sync(0xffffffffu, badnan, o);
    quiet += __shfl_down_sync(0xffffffffu, quiet, o);
  }
  if ((threadIdx.x & 31) == 0 && (bad | badnan | quiet)) {
    atomicAdd(&g_promote_mismatch[0], bad);
    atomicAdd(&g_promote_mismatch[1], badnan);
    atomicAdd(&g_promote_mismatch[2], quiet);
  }
}

}  // namespace
}  // namespace gbs

extern "C" gbs_status gbs_selftest_f32_to_f64(uint64_t first, uint64_t count, uint64_t* mismatches) {
  if (!mismatches || first > (1ull << 32) || count > (1ull << 32) - first) return GBS_ERR_INVALID;
  const unsigned long long zero[3] = {0, 0, 0};
  if (cudaMemcpyToSymbol(gbs::g_promote_mismatch, zero, sizeof zero) != cudaSuccess) return GBS_ERR_CUDA;
  if (count) {
    gbs::k_selftest_promote<<<4096, 256>>>(first, count);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return GBS_ERR_CUDA;
  }
  unsigned long long out[3];
  if (cudaMemcpyFromSymbol(out, gbs::g_promote_mismatch, sizeof out) != cudaSuccess) return GBS_ERR_CUDA;
  for (int i = 0; i < 3; ++i) mismatches[i] = out[i];
  return GBS_OK;
}
