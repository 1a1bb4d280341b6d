// k_resample.cu -- resampling of series for the frequency derivatives f1,
// f2 of a periodic signal (Sec.3.4), so that a signal of frequency
// f0 + f1 t + f2 t^2/2 comes out at a constant frequency.
//
// Output bin k has width w_k = tau_k / tau0 = 1 + alpha k + beta k^2 input
// samples (the Doppler interval tau = tau0 (1 + f' t/f0 + f'' t^2/(2 f0))
// at the bin's nominal time t = k tau0, alpha = f' tau0/f0,
// beta = f'' tau0^2/(2 f0)), so its start is the closed form
//   t_k = k + alpha k(k-1)/2 + beta (k-1)k(2k-1)/6
// and every bin is computed on its own: out[k] sums the one to three input
// samples it overlaps, each weighted by the overlap (FP64 arithmetic, FP32
// result).  f1 > 0 reverses the series, uses f0~ = f0 + f1 T + f2 T^2/2,
// f' = f1 + f2 T, f'' = -f2, and reverses the result; f1 <= 0 uses f0,
// f' = -f1, f'' = -f2.
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "host.h"

namespace ddsp {
namespace {

struct ResampleLaw {
  double alpha, beta;   // bin width 1 + alpha k + beta k^2 (input samples)
  bool rev;             // f1 > 0: work on the reversed series
  bool ok;
};

ResampleLaw resample_law(int64_t n, double tsamp, double f0, double f1,
                         double f2) {
  ResampleLaw L{0.0, 0.0, false, false};
  if (n < 1 || !(tsamp > 0.0) || !(f0 > 0.0) || !std::isfinite(f1) ||
      !std::isfinite(f2))
    return L;
  const double T = (double)n * tsamp;
  double F0 = f0, fp = -f1, fpp = -f2;
  if (f1 > 0.0) {
    F0 = f0 + f1 * T + f2 * T * T / 2.0;
    fp = f1 + f2 * T;
    fpp = -f2;
    L.rev = true;
    if (!(F0 > 0.0)) return L;
  }
  L.alpha = fp * tsamp / F0;
  L.beta = fpp * tsamp * tsamp / (2.0 * F0);
  L.ok = true;
  return L;
}

__host__ __device__ __forceinline__ double bin_start(double k, double a,
                                                     double b) {
  return k + a * k * (k - 1.0) / 2.0 + b * (k - 1.0) * k * (2.0 * k - 1.0) / 6.0;
}

// Bins kept: the largest K with t_K <= n while every width is > 0; -1 if a
// width before that is <= 0.
int64_t resample_count(int64_t n, const ResampleLaw &L) {
  // widths stay near 1 for real laws: bins that cannot cover the series
  // within 2n + 16 of them (average width below about 1/2) are refused
  int64_t lo = 0, hi = 2 * n + 16;
  if (bin_start((double)hi, L.alpha, L.beta) <= (double)n) return -1;
  auto width = [&](double k) { return 1.0 + L.alpha * k + L.beta * k * k; };
  // the largest K with t_K <= n among K where all widths so far are > 0
  while (hi - lo > 1) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (bin_start((double)mid, L.alpha, L.beta) <= (double)n) lo = mid;
    else hi = mid;
  }
  const int64_t K = lo;
  if (K > 0) {
    // widths 0 .. K-1 are > 0: check the ends and the vertex of the parabola
    double wmin = std::min(width(0.0), width((double)(K - 1)));
    if (L.beta != 0.0) {
      const double kv = -L.alpha / (2.0 * L.beta);
      if (kv > 0.0 && kv < (double)(K - 1)) wmin = std::min(wmin, width(kv));
    }
    if (!(wmin > 0.0)) return -1;
  }
  return K;
}

__global__ void resample_kernel(const int32_t *__restrict__ in, int64_t nrows,
                                int64_t n, int64_t in_pitch, double a, double b,
                                bool rev, int64_t K, float *__restrict__ out,
                                int64_t out_pitch) {
  const int64_t total = nrows * K;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
       idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / K, k = idx - r * K;
    const double t0 = bin_start((double)k, a, b);
    const double t1 = bin_start((double)(k + 1), a, b);
    const int32_t *x = in + r * in_pitch;
    double acc = 0.0;
    const int64_t i0 = (int64_t)floor(t0), i1 = (int64_t)floor(t1);
    for (int64_t i = max(i0, (int64_t)0); i <= i1 && i < n; ++i) {
      const double lo = fmax(t0, (double)i), hi = fmin(t1, (double)(i + 1));
      if (hi > lo) acc += (double)x[rev ? n - 1 - i : i] * (hi - lo);
    }
    out[r * out_pitch + (rev ? K - 1 - k : k)] = (float)acc;
  }
}

}  // namespace
}  // namespace ddsp

using namespace ddsp;

extern "C" int ddsp_resample_length(int64_t nsamp, double tsamp, double f0,
                                    double f1, double f2, int64_t *nout) {
  if (!nout) return DDSP_E_INVALID_ARG;
  const ResampleLaw L = resample_law(nsamp, tsamp, f0, f1, f2);
  if (!L.ok) return DDSP_E_INVALID_ARG;
  const int64_t K = resample_count(nsamp, L);
  if (K < 0) return DDSP_E_INVALID_ARG;
  *nout = K;
  return DDSP_OK;
}

extern "C" int ddsp_resample(ddsp_plan *h, const int32_t *d_in, int64_t nrows,
                             int64_t nsamp, int64_t in_pitch, double tsamp,
                             double f0, double f1, double f2, float *d_out,
                             int64_t out_pitch, int64_t *nout,
                             ddsp_stream_t stream) {
  if (!h || !d_in || !nout || nrows <= 0 || in_pitch < nsamp)
    return DDSP_E_INVALID_ARG;
  const ResampleLaw L = resample_law(nsamp, tsamp, f0, f1, f2);
  if (!L.ok) return DDSP_E_INVALID_ARG;
  const int64_t K = resample_count(nsamp, L);
  if (K < 0 || out_pitch < K || (K > 0 && !d_out)) return DDSP_E_INVALID_ARG;
  *nout = K;
  if (K == 0) return DDSP_OK;
  DeviceGuard g(h->p.device);
  const int64_t total = nrows * K;
  const int64_t blocks = std::min<int64_t>((total + 255) / 256, 148 * 32);
  resample_kernel<<<(unsigned)blocks, 256, 0,
                    reinterpret_cast<cudaStream_t>(stream)>>>(
      d_in, nrows, nsamp, in_pitch, L.alpha, L.beta, L.rev, K, d_out,
      out_pitch);
  return cuda_rc(cudaGetLastError());
}
