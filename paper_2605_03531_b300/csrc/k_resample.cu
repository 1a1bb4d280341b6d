// k_resample.cu -- resampling of series for the frequency derivatives f1,
// f2 of a periodic signal (Sec.3.4), so that a signal of frequency
// f0 + f1 t + f2 t^2/2 comes out at a constant frequency.
//
// Output bin k has width w_k = tau_k / tau0 = 1 + alpha k + beta k^2 input
// samples (the Doppler interval tau = tau0 (1 + f' t/f0 + f'' t^2/(2 f0))
// at the bin's nominal time t = k tau0, alpha = f' tau0/f0,
// beta = f'' tau0^2/(2 f0)), so its start is the closed form
//   t_k = k + alpha k(k-1)/2 + beta (k-1)k(2k-1)/6
// and out[k] sums the one to three input samples the bin overlaps, each
// weighted by the overlap (FP32, relative to an exact integer sample index
// taken every 32 bins from the FP64 closed form, which the host tabulates:
// the device does no FP64 arithmetic).  f1 > 0 reverses the series, uses
// f0~ = f0 + f1 T + f2 T^2/2,
// f' = f1 + f2 T, f'' = -f2, and reverses the result; f1 <= 0 uses f0,
// f' = -f1, f'' = -f2.
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

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

inline double bin_start(double k, double a, double b) {
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

constexpr int kRsGroups = 32;

// First edge of a group of 32 bins: t_{32g} = ib + fr, ib an integer sample
// index and 0 <= fr < 1 (FP64 on the host, fr rounded to FP32 once).
struct RsEdge {
  long long ib;
  float fr;
  int pad;
};

// A warp makes kRsGroups groups of 32 consecutive bins, one bin per lane:
// lane l first loads group l's first edge (tabulated on the host in FP64),
// then per group a warp prefix sum of the bins' FP32 width deviations from
// one sample places lane l's bin at ib + l + e, and the overlaps are
// computed from the bin's own integer sample, so every FP32 value stays
// near 1 (edge error about 2^-22 samples) and the lanes read and write
// consecutive samples.
__global__ void resample_kernel(const int32_t *__restrict__ in, int64_t nrows,
                                int64_t n, int64_t in_pitch, float af, float bf,
                                const RsEdge *__restrict__ edges, bool rev,
                                int64_t K, float *__restrict__ out,
                                int64_t out_pitch) {
  const int lane = threadIdx.x & 31;
  const int64_t groups = (K + 31) / 32;            // 32 bins each
  const int64_t supers = (groups + kRsGroups - 1) / kRsGroups;
  const int64_t total = nrows * supers;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t sg = w0; sg < total; sg += nw) {
    const int64_t r = sg / supers, g0 = (sg - r * supers) * kRsGroups;
    // lane l: the first edge of group g0 + l
    long long ibl = 0;
    float frl = 0.0f;
    if (g0 + lane < groups) {
      const RsEdge ed = edges[g0 + lane];
      ibl = ed.ib;
      frl = ed.fr;
    }
    const int32_t *x = in + r * in_pitch;
    const int gn = (int)min((int64_t)kRsGroups, groups - g0);
    for (int q = 0; q < gn; ++q) {
      const long long ib = __shfl_sync(0xffffffffu, ibl, q);
      const float fr = __shfl_sync(0xffffffffu, frl, q);
      const int64_t k = (g0 + q) * 32 + lane;
      const float kf = (float)k;
      // width deviation from one sample (small), and its exclusive prefix
      const float dev = k < K ? af * kf + bf * kf * kf : 0.0f;
      float incl = dev;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const float u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
      }
      if (k >= K) continue;
      // the bin starts lane + e samples after ib; counted from its own
      // integer sample it spans [f, f + 1 + dev): every value stays near 1
      const float e = fr + (incl - dev);
      const float fl = floorf(e);
      const float f = e - fl, fe = f + 1.0f + dev;
      const int64_t base = ib + lane + (int64_t)fl;
      float acc = 0.0f;
      // the first two overlap terms unrolled (their loads issue together),
      // then bins wider than two samples; same order of terms as a loop
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        const float lo = fmaxf(f, (float)d), hi = fminf(fe, (float)(d + 1));
        const int64_t i = base + d;
        if (hi > lo && i >= 0 && i < n)
          acc += (float)x[rev ? n - 1 - i : i] * (hi - lo);
      }
      for (int d = 2; (float)d < fe && base + d < n; ++d) {
        const float lo = fmaxf(f, (float)d), hi = fminf(fe, (float)(d + 1));
        const int64_t i = base + d;
        if (hi > lo && i >= 0) acc += (float)x[rev ? n - 1 - i : i] * (hi - lo);
      }
      out[r * out_pitch + (rev ? K - 1 - k : k)] = acc;
    }
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
  Plan &p = h->p;
  // every group's first edge, from the FP64 closed form on the host
  const int64_t groups = (K + 31) / 32;
  std::vector<RsEdge> edges((size_t)groups);
  for (int64_t q = 0; q < groups; ++q) {
    const double t0 = bin_start((double)(q * 32), L.alpha, L.beta);
    const double fl = floor(t0);
    edges[(size_t)q].ib = (long long)fl;
    edges[(size_t)q].fr = (float)(t0 - fl);
    edges[(size_t)q].pad = 0;
  }
  const size_t bytes = (size_t)groups * sizeof(RsEdge);
  if (bytes > p.rs_bytes) {
    cudaDeviceSynchronize();   // a previous call may still read the table
    cudaFree(p.d_rs);
    p.d_rs = nullptr;
    p.rs_bytes = 0;
    cudaError_t e = cudaMalloc(&p.d_rs, bytes);
    if (e != cudaSuccess) return cuda_rc(e);
    p.rs_bytes = bytes;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // from pageable memory: the call returns once the table has been staged,
  // and the copy is ordered before the kernel on the same stream
  cudaError_t e = cudaMemcpyAsync(p.d_rs, edges.data(), bytes,
                                  cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_rc(e);
  const int64_t total =
      nrows * ((groups + kRsGroups - 1) / kRsGroups);      // warps
  const int64_t blocks = std::min<int64_t>((total + 7) / 8, 148 * 32);
  resample_kernel<<<(unsigned)blocks, 256, 0, s>>>(
      d_in, nrows, nsamp, in_pitch, (float)L.alpha, (float)L.beta,
      static_cast<const RsEdge *>(p.d_rs), L.rev, K, d_out, out_pitch);
  return cuda_rc(cudaGetLastError());
}
