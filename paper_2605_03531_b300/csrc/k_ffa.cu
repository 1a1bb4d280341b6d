// k_ffa.cu -- the folding transform by the fast folding algorithm and the
// boxcar search of the folded profiles (Sec.3.5), for rows of int32 series.
//
// One block per (row, base period p): the first m*p samples of the row
// (m the largest power of two with m*p <= nsamp) are loaded into shared
// memory and transformed in log2(m) levels between two buffers; at the
// level merging groups of n rows, output profile s of a group is
//   F[s][j] = A[s/2][j] + B[s/2][(j + (s+1)/2) mod p],
// A and B the transforms of the group's two halves (the classic binary
// recursion: profile s drifts by s samples over the m - 1 row steps, i.e.
// trial period p + s/(m - 1)).  Sums are int32, checked on every add.
//
// The search gives one warp to each profile: it writes the profile's
// exclusive prefix sums (mod 2^32) into the spare transform buffer, and when
// every boxcar sum of the profile fits int32 (w_max * max|P| < 2^31) a
// cyclic boxcar is a difference of two of them; otherwise the lanes extend
// running int64 window sums.  The numerator p*B - w*S of
// S/N = (B - w*S/p) / (sigma*sqrt(m*w)) is exact in int64 and rounded to
// FP32 once (hi/lo split, magic-number conversion, one fma), then scaled by
// the width's 1/(p sigma sqrt(m w)); the largest S/N wins, ties to the
// smaller width, then the smaller phase.
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "host.h"

namespace ddsp {
namespace {

constexpr int kFfaThreads = 1024;
constexpr int kFfaMaxStack = 16384;        // m * p per block (shared memory)
constexpr int kFfaMaxWidths = 16;

struct FfaWidths {
  int32_t w[kFfaMaxWidths];
  int n;
};

// float(v) rounded once, for |v| < 2^43 (two exact magic-number
// conversions of 22-bit halves and one fused multiply-add)
__device__ __forceinline__ float i64_to_float(long long v) {
  const int32_t hi = (int32_t)(v >> 21);
  const int32_t lo = (int32_t)(v & 0x1FFFFF);
  const float magic = 12582912.0f;            // 1.5 * 2^23
  const float hf = __int_as_float(0x4B400000 + hi) - magic;
  const float lf = __int_as_float(0x4B400000 + lo) - magic;
  return __fmaf_rn(hf, 2097152.0f, lf);
}

// Transform the stack in buf0 (m rows of p); returns the buffer holding the
// result.  One warp per output row, lanes along the row: the row's sources
// and shift are found once per row.
__device__ int32_t *ffa_levels(int32_t *buf0, int32_t *buf1, int p, int m,
                               int32_t *err) {
  int32_t *src = buf0, *dst = buf1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  for (int lg = 1; (1 << lg) <= m; ++lg) {
    const int n = 1 << lg, half = n >> 1;
    bool bad = false;
    for (int row = warp; row < m; row += nwarps) {
      const int g = row >> lg, s = row & (n - 1);
      const int a = s >> 1;
      const int sh = ((s + 1) >> 1) % p;
      const int32_t *A = src + (g * n + a) * p;
      const int32_t *B = src + (g * n + half + a) * p;
      int32_t *D = dst + row * p;
      for (int j = lane; j < p; j += 32) {
        int jj = j + sh;
        if (jj >= p) jj -= p;
        const int32_t u = A[j], w = B[jj];
        const int32_t v = (int32_t)((uint32_t)u + (uint32_t)w);
        bad |= ((u ^ v) & (w ^ v)) < 0;      // signed overflow of u + w
        D[j] = v;
      }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicExch(err, kErrRange);
    __syncthreads();
    int32_t *t = src;
    src = dst;
    dst = t;
  }
  return src;
}

__device__ __forceinline__ int ffa_rows(int64_t nsamp, int p) {
  int m = 1;
  while ((int64_t)2 * m * p <= nsamp) m *= 2;
  return m;
}

__global__ void __launch_bounds__(kFfaThreads)
ffa_kernel(const int32_t *__restrict__ in, int64_t nsamp, int64_t pitch, int p,
           int32_t *__restrict__ out, int32_t *err) {
  extern __shared__ __align__(16) int32_t sm[];
  const int m = ffa_rows(nsamp, p);
  const int total = m * p;
  int32_t *buf0 = sm, *buf1 = sm + total;
  const int32_t *x = in + (int64_t)blockIdx.x * pitch;
  for (int i = threadIdx.x; i < total; i += blockDim.x) buf0[i] = x[i];
  __syncthreads();
  const int32_t *F = ffa_levels(buf0, buf1, p, m, err);
  int32_t *o = out + (int64_t)blockIdx.x * total;
  for (int i = threadIdx.x; i < total; i += blockDim.x) o[i] = F[i];
}

__global__ void __launch_bounds__(kFfaThreads)
ffa_search_kernel(const int32_t *__restrict__ in, int64_t nsamp, int64_t pitch,
                  int p_lo, FfaWidths W, const float *__restrict__ sigma,
                  float *__restrict__ snr_out, int32_t *__restrict__ w_out,
                  int32_t *__restrict__ ph_out, int64_t mmax, int32_t *err) {
  extern __shared__ __align__(16) int32_t sm[];
  const int p = p_lo + blockIdx.x;
  const int64_t row = blockIdx.y;
  const int m = ffa_rows(nsamp, p);
  const int total = m * p;
  int32_t *buf0 = sm, *buf1 = sm + total;
  const int32_t *x = in + row * pitch;
  for (int i = threadIdx.x; i < total; i += blockDim.x) buf0[i] = x[i];
  __syncthreads();
  const int32_t *F = ffa_levels(buf0, buf1, p, m, err);

  int32_t *spare = F == buf0 ? buf1 : buf0;   // profiles' prefix sums
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  // widths that fit the profile, and their FP32 scales 1/(p sigma sqrt(m w))
  int nw = 0;
  while (nw < W.n && W.w[nw] <= p) ++nw;
  const int wmax = nw > 0 ? W.w[nw - 1] : 0;
  const float sg = sigma[row];
  __shared__ float inv[kFfaMaxWidths];
  if (threadIdx.x < kFfaMaxWidths)
    inv[threadIdx.x] = (int)threadIdx.x < nw
        ? 1.0f / (p * sg * sqrtf((float)m * (float)W.w[threadIdx.x])) : 0.0f;
  __syncthreads();
  const int64_t obase = (row * gridDim.x + blockIdx.x) * mmax;
  for (int s = warp; s < (int)mmax; s += nwarps) {
    if (s >= m || nw == 0) {
      if (lane == 0) {
        snr_out[obase + s] = -INFINITY;
        w_out[obase + s] = -1;
        ph_out[obase + s] = -1;
      }
      continue;
    }
    const int32_t *P = F + s * p;
    uint32_t *Q = reinterpret_cast<uint32_t *>(spare) + s * p;
    // exclusive prefix sums (mod 2^32), the total and the largest |P|
    long long S = 0;
    uint32_t run = 0, amax = 0;
    for (int j0 = 0; j0 < p; j0 += 32) {
      const int j = j0 + lane;
      const int32_t v = j < p ? P[j] : 0;
      amax = max(amax, v < 0 ? 0u - (uint32_t)v : (uint32_t)v);
      S += v;
      uint32_t inc = (uint32_t)v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
      }
      if (j < p) Q[j] = run + inc - (uint32_t)v;
      run += __shfl_sync(0xffffffffu, inc, 31);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      S += __shfl_xor_sync(0xffffffffu, S, o);
      amax = max(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    }
    __syncwarp();
    // every boxcar sum fits int32, so prefix differences mod 2^32 are exact
    const bool fast = (unsigned long long)amax * (unsigned long long)wmax <
                      0x80000000ull;
    const uint32_t Sq = (uint32_t)S;
    float best = -INFINITY;
    int bw = 0, bj = 0;
    for (int j = lane; j < p; j += 32) {
      if (fast) {
        const uint32_t q0 = Q[j];
        for (int wi = 0; wi < nw; ++wi) {
          const int e = j + W.w[wi];
          const uint32_t q1 = e < p ? Q[e] : Sq + Q[e - p];
          const int32_t B = (int32_t)(q1 - q0);
          const long long num = (long long)p * B - (long long)W.w[wi] * S;
          const float nf = (num < (1ll << 43) && num > -(1ll << 43))
                               ? i64_to_float(num) : __ll2float_rn(num);
          const float sn = nf * inv[wi];
          if (sn > best || (sn == best && (wi < bw || (wi == bw && j < bj)))) {
            best = sn;
            bw = wi;
            bj = j;
          }
        }
      } else {
        long long B = 0;
        int wi = 0, jj = j;
        for (int i = 0; i < wmax; ++i) {
          B += P[jj];
          if (++jj == p) jj = 0;
          if (i + 1 == W.w[wi]) {
            const long long num = (long long)p * B - (long long)W.w[wi] * S;
            const float nf = (num < (1ll << 43) && num > -(1ll << 43))
                                 ? i64_to_float(num) : __ll2float_rn(num);
            const float sn = nf * inv[wi];
            if (sn > best || (sn == best && (wi < bw || (wi == bw && j < bj)))) {
              best = sn;
              bw = wi;
              bj = j;
            }
            ++wi;
          }
        }
      }
    }
    // ties go to the smaller width, then the smaller phase, within and
    // across lanes
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int ow = __shfl_xor_sync(0xffffffffu, bw, o);
      const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
      if (ob > best || (ob == best && (ow < bw || (ow == bw && oj < bj)))) {
        best = ob;
        bw = ow;
        bj = oj;
      }
    }
    if (lane == 0) {
      snr_out[obase + s] = best;
      w_out[obase + s] = bw;
      ph_out[obase + s] = bj;
    }
  }
}

int host_ffa_rows(int64_t nsamp, int p) {
  if (p < 1 || nsamp < p) return 0;
  int m = 1;
  while ((int64_t)2 * m * p <= nsamp) m *= 2;
  return m;
}

}  // namespace
}  // namespace ddsp

using namespace ddsp;

extern "C" int ddsp_ffa(ddsp_plan *h, const int32_t *d_series, int64_t nrows,
                        int64_t nsamp, int64_t pitch, int p, int32_t *d_out,
                        int *m_out, ddsp_stream_t stream) {
  if (!h || !d_series || !d_out || !m_out || nrows <= 0 || nrows > 65535 * 32 ||
      pitch < nsamp)
    return DDSP_E_INVALID_ARG;
  const int m = host_ffa_rows(nsamp, p);
  if (m == 0 || (int64_t)m * p > kFfaMaxStack) return DDSP_E_INVALID_ARG;
  *m_out = m;
  DeviceGuard g(h->p.device);
  const size_t smem = (size_t)2 * m * p * 4;
  cudaError_t e = smem_opt_in(ffa_kernel);
  if (e != cudaSuccess) return cuda_rc(e);
  ffa_kernel<<<(unsigned)nrows, kFfaThreads, smem,
               reinterpret_cast<cudaStream_t>(stream)>>>(d_series, nsamp, pitch,
                                                         p, d_out, h->p.d_err);
  return cuda_rc(cudaGetLastError());
}

extern "C" int ddsp_ffa_search(ddsp_plan *h, const int32_t *d_series,
                               int64_t nrows, int64_t nsamp, int64_t pitch,
                               int p_lo, int p_hi, const int32_t *widths,
                               int nwidths, const float *d_sigma, float *d_snr,
                               int32_t *d_widx, int32_t *d_phase, int64_t mmax,
                               ddsp_stream_t stream) {
  if (!h || !d_series || !widths || !d_sigma || !d_snr || !d_widx ||
      !d_phase || nrows <= 0 || nrows > 65535 || pitch < nsamp || p_lo < 1 ||
      p_hi <= p_lo || nwidths < 1 || nwidths > kFfaMaxWidths)
    return DDSP_E_INVALID_ARG;
  FfaWidths W{};
  W.n = nwidths;
  for (int i = 0; i < nwidths; ++i) {
    W.w[i] = widths[i];
    if (widths[i] < 1 || (i > 0 && widths[i] <= widths[i - 1]))
      return DDSP_E_INVALID_ARG;
  }
  int mlo = host_ffa_rows(nsamp, p_lo);
  if (mlo == 0 || mmax < mlo || host_ffa_rows(nsamp, p_hi - 1) == 0)
    return DDSP_E_INVALID_ARG;
  size_t smem = 0;
  for (int p = p_lo; p < p_hi; ++p) {
    const int64_t st = (int64_t)host_ffa_rows(nsamp, p) * p;
    if (st > kFfaMaxStack) return DDSP_E_INVALID_ARG;
    smem = std::max(smem, (size_t)(2 * st * 4));
  }
  DeviceGuard g(h->p.device);
  cudaError_t e = smem_opt_in(ffa_search_kernel);
  if (e != cudaSuccess) return cuda_rc(e);
  dim3 grid((unsigned)(p_hi - p_lo), (unsigned)nrows);
  ffa_search_kernel<<<grid, kFfaThreads, smem,
                      reinterpret_cast<cudaStream_t>(stream)>>>(
      d_series, nsamp, pitch, p_lo, W, d_sigma, d_snr, d_widx, d_phase, mmax,
      h->p.d_err);
  return cuda_rc(cudaGetLastError());
}
