// The one-way wave u_t + u_x = 0 with a spectral derivative (Sec. 4), FP64.
//
// A problem has n <= 2048 points, so one block holds a whole macro-step in shared memory: the
// state y_0, the shared first evaluation f0 = f(y_0) (Sec. 3.6), the two leap-frog levels of
// the current sequence, the evaluation scratch and the FP64 combine accumulator.  Every right-
// hand-side evaluation is a radix-2 FFT of the level (a real signal, as one complex FFT of half
// the length), a multiplication of mode m by -i k_m (k_m = 2 pi m / (n dx),
// m = -n/2+1 .. n/2-1; the Nyquist mode, whose derivative the grid cannot represent, set to
// zero) and an inverse FFT (Sec. 4: spectral derivatives, so the
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

// In-place radix-2 decimation-in-time FFT of z[0..m) (m = 2^logm): bit-reversal permutation,
// then logm butterfly stages.  tw[q] = exp(-2 pi i q / n), q < n/2, is the table of a length-n
// transform, n = tmul m: stage s takes exp(-2 pi i pos / 2^s) = tw[pos (m >> s) tmul].  Inverse =
// conjugate twiddles, unscaled.  Ends with a barrier.
__device__ void fft(double2* z, const double2* tw, int m, int logm, int tmul, bool inverse) {
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const int j = (int)(__brev((unsigned)i) >> (32 - logm));
    if (i < j) {
      const double2 t = z[i];
      z[i] = z[j];
      z[j] = t;
    }
  }
  __syncthreads();
  for (int s = 1; s <= logm; ++s) {
    const int half = 1 << (s - 1);
    const int tstride = (m >> s) * tmul;
    for (int b = threadIdx.x; b < m / 2; b += blockDim.x) {
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

// f = -u_x spectrally (the header above), u real of length n: the transform of a real signal as
// one complex transform of half the length (the even samples as real parts, the odd ones as
// imaginary parts), so each derivative costs two length-n/2 FFTs.  With m = n/2, Z = FFT_m(z)
// and W = exp(-2 pi i / n), the real signal's bins are U_k = E_k + W^k O_k and
// U_(m-k) = conj(E_k - W^k O_k), where E_k = (Z_k + conj Z_(m-k)) / 2 and
// O_k = (Z_k - conj Z_(m-k)) / (2i); the derivative's bins F = -i k_m U (zero at k = 0 and at the
// Nyquist bin m) go back the same way, Z'_k = (F_k + conj F_(m-k)) / 2 +
// i (F_k - conj F_(m-k)) conj(W^k) / 2 and Z'_(m-k) from the conjugates, and the inverse
// FFT_m of Z' holds f's even and odd samples, times m.  One thread takes the bins k and m - k
// together, so the update is in place.  u and f in shared memory, z scratch (n/2 entries).
// Ends with a barrier.
__device__ void spectral_rhs(const double* u, double* f, double2* z, const double2* tw, int n, int logn,
                             double kscale) {
  const int m = n >> 1, logm = logn - 1;
  for (int j = threadIdx.x; j < m; j += blockDim.x) z[j] = make_double2(u[2 * j], u[2 * j + 1]);
  __syncthreads();
  fft(z, tw, m, logm, 2, false);
  for (int k = threadIdx.x; k <= m / 2; k += blockDim.x) {
    if (k == 0) {
      z[0] = make_double2(0.0, 0.0);   // the mean and the Nyquist mode have derivative zero
      continue;
    }
    const int kp = m - k;
    const double2 a = z[k], b = z[kp], w = tw[k];
    const double2 e = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
    const double2 o = make_double2(0.5 * (a.y + b.y), -0.5 * (a.x - b.x));
    const double2 wo = cmul(w, o);
    const double2 uk = make_double2(e.x + wo.x, e.y + wo.y);
    const double2 ukp = make_double2(e.x - wo.x, -(e.y - wo.y));
    const double sk = kscale * (double)k, skp = kscale * (double)kp;
    const double2 fk = make_double2(sk * uk.y, -sk * uk.x);        // -i k U
    const double2 fkp = make_double2(skp * ukp.y, -skp * ukp.x);
    const double2 ef = make_double2(0.5 * (fk.x + fkp.x), 0.5 * (fk.y - fkp.y));
    const double2 of = cmul(make_double2(0.5 * (fk.x - fkp.x), 0.5 * (fk.y + fkp.y)), make_double2(w.x, -w.y));
    z[k] = make_double2(ef.x - of.y, ef.y + of.x);
    if (kp != k) z[kp] = make_double2(ef.x + of.y, -ef.y + of.x);
  }
  __syncthreads();
  fft(z, tw, m, logm, 2, true);
  const double inv_m = 1.0 / (double)m;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    f[2 * j] = z[j].x * inv_m;
    f[2 * j + 1] = z[j].y * inv_m;
  }
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
