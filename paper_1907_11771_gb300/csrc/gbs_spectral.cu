// The one-way wave u_t + u_x = 0 with a spectral derivative (Sec. 4), FP64.
//
// A problem has n <= 2048 points, so one block holds a whole macro-step in shared memory: the
// state y_0, the shared first evaluation f0 = f(y_0) (Sec. 3.6), the two leap-frog levels of
// the current sequence, the evaluation scratch and the FP64 combine accumulator.  Every right-
// hand-side evaluation is a radix-2 FFT of the level, a multiplication of mode m by
// -i k_m (k_m = 2 pi m / (n dx), m = -n/2+1 .. n/2-1; the Nyquist mode, whose derivative the
// grid cannot represent, set to zero) and an inverse FFT (Sec. 4: spectral derivatives, so the
// errors are the time stepper's).  Then, per sequence k with h = H / N_k (eq. "GBS"): Forward
// Euler from f0, N_k leap-frog steps, the average (y_(N-1) + 2 y_N + y_(N+1)) / 4, and
// y_out = sum_k c_k y*_k accumulated in FP64 (Sec. 2.1, Sec. 3.2).  One block per problem.
#include <cuda_runtime.h>

#include <cmath>

#include "gbs_internal.h"

namespace gbs {
namespace {

constexpr int kSpecThreads = 512;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// In-place radix-2 decimation-in-time FFT of z[0..n) (n = 2^logn): bit-reversal permutation,
// then logn butterfly stages.  tw[m] = exp(-2 pi i m / n), m < n/2; inverse = conjugate
// twiddles, unscaled.  Ends with a barrier.
__device__ void fft(double2* z, const double2* tw, int n, int logn, bool inverse) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int j = (int)(__brev((unsigned)i) >> (32 - logn));
    if (i < j) {
      const double2 t = z[i];
      z[i] = z[j];
      z[j] = t;
    }
  }
  __syncthreads();
  for (int s = 1; s <= logn; ++s) {
    const int half = 1 << (s - 1);
    const int tstride = n >> s;
    for (int b = threadIdx.x; b < n / 2; b += blockDim.x) {
      const int pos = b & (half - 1);
      const int i = ((b >> (s - 1)) << s) + pos;
      double2 w = tw[pos * tstride];
      if (inverse) w.y = -w.y;
      const double2 t = cmul(w, z[i + half]);
      const double2 a = z[i];
      z[i] = make_double2(a.x + t.x, a.y + t.y);
      z[i + half] = make_double2(a.x - t.x, a.y - t.y);
    }
    __syncthreads();
  }
}

// f = -u_x spectrally (the header above); u and f in shared memory, z scratch.  Ends with a barrier.
__device__ void spectral_rhs(const double* u, double* f, double2* z, const double2* tw, int n, int logn,
                             double kscale) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) z[i] = make_double2(u[i], 0.0);
  __syncthreads();
  fft(z, tw, n, logn, false);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int m = i < n / 2 ? i : (i == n / 2 ? 0 : i - n);
    const double k = kscale * (double)m;
    const double2 a = z[i];
    z[i] = make_double2(k * a.y, -k * a.x);   // (a.x + i a.y) * (-i k)
  }
  __syncthreads();
  fft(z, tw, n, logn, true);
  const double inv_n = 1.0 / (double)n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) f[i] = z[i].x * inv_n;
  __syncthreads();
}

__global__ void __launch_bounds__(kSpecThreads) k_spectral_macro(const StepPlan p, const double* y_in,
                                                                 double* y_out) {
  extern __shared__ double sm[];
  const int prob = blockIdx.x;
  const ProbDev& q = p.probs[prob];
  const SlotDev& s = p.slots[q.slot];
  const int n = q.n[0];
  const int logn = 31 - __clz(n);
  double* y0 = sm;
  double* f0 = y0 + n;
  double* la = f0 + n;
  double* lb = la + n;
  double* fe = lb + n;
  double* acc = fe + n;
  double2* z = reinterpret_cast<double2*>(acc + n);
  double2* tw = z + n;
  for (int m = threadIdx.x; m < n / 2; m += blockDim.x) {
    double sn, cs;
    sincospi(2.0 * (double)m / (double)n, &sn, &cs);
    tw[m] = make_double2(cs, -sn);
  }
  const double* yi = y_in + q.state_off;
  for (int i = threadIdx.x; i < n; i += blockDim.x) y0[i] = yi[i];
  __syncthreads();
  const double kscale = 2.0 * M_PI * q.inv_dx[0] / (double)n;
  spectral_rhs(y0, f0, z, tw, n, logn, kscale);
  for (int k = 0; k < s.m; ++k) {
    const int N = s.steps[k];
    const double h = p.hk[prob * GBS_MAX_SEQ + k];
    const double h2 = 2.0 * h;
    const double c = s.c[k];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      la[i] = y0[i];
      lb[i] = fma(h, f0[i], y0[i]);   // Forward Euler y_1
    }
    __syncthreads();
    double* ym = la;   // y_(j-1)
    double* yc = lb;   // y_j
    for (int j = 1; j <= N; ++j) {
      spectral_rhs(yc, fe, z, tw, n, logn, kscale);
      if (j < N) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) ym[i] = fma(h2, fe[i], ym[i]);   // y_(j+1)
        __syncthreads();
        double* t = ym;
        ym = yc;
        yc = t;
      } else {
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
          const double yp = fma(h2, fe[i], ym[i]);
          const double ys = (ym[i] + 2.0 * yc[i] + yp) * 0.25;
          acc[i] = k == 0 ? c * ys : fma(c, ys, acc[i]);
        }
        __syncthreads();
      }
    }
  }
  double* yo = y_out + q.state_off;
  for (int i = threadIdx.x; i < n; i += blockDim.x) yo[i] = acc[i];
}

size_t spectral_smem(int n) { return (size_t)n * (6 * sizeof(double) + sizeof(double2)) + (size_t)(n / 2) * sizeof(double2); }

}  // namespace

int spectral_setup() {
  const cudaError_t e = cudaFuncSetAttribute(k_spectral_macro, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)spectral_smem(kSpectralMaxN));
  return e == cudaSuccess ? 0 : -1;
}

int spectral_macro_step(const StepPlan& p, const void* y_in, void* y_out, cudaStream_t st) {
  k_spectral_macro<<<p.batch, kSpecThreads, spectral_smem((int)p.max_nx), st>>>(p, static_cast<const double*>(y_in),
                                                                             static_cast<double*>(y_out));
  return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace gbs
