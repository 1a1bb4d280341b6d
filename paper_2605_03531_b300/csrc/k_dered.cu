// k_dered.cu -- downsampling of dedispersed series by a user factor
// (Sec.3.2) and running-median de-reddening (Sec.3.3), on rows of int32
// series in device memory.
//
// Downsampling: y[j] = sum_{i<f} x[j*f + i] in int64, checked against the
// int32 range (the plan's error word records DDSP_E_RANGE); one thread per
// output for f < 32, one warp per output (lanes stride the group, shuffle
// reduction) otherwise.
//
// De-reddening: z[t] = x[t] - m[t], m[t] the lower median of x over
// [t - h, t + h] clamped to the row.  One block per (row, chunk of T
// outputs) loads the chunk's span [t0 - h, t0 + T + h) (clamped) into
// shared memory and builds a wavelet matrix of its values relative to the
// span's minimum: level l splits the values by bit (L - 1 - l), MSB first,
// keeping order within each side (zeros first); per level a bit word per 32
// positions (warp ballots), their exclusive popcount prefix (one block
// scan) and the zero count.  The median of any window of the span is then
// a k-th-smallest query answered in L steps of two popcount ranks each, so
// every output is computed independently, exactly (ties included), with no
// per-window sort.  Shared memory: 8 B per span element for the two
// partition buffers plus, per level, a bit word and a prefix word per 32
// elements.
#include <stdint.h>

#include <algorithm>

#include "host.h"

namespace ddsp {
namespace {

constexpr int kDsThreads = 256;
constexpr int kDrThreads = 512;
constexpr int kDrMaxLevels = 32;

__global__ void downsample_thread_kernel(const int32_t *__restrict__ in,
                                         int64_t nrows, int64_t m,
                                         int64_t in_pitch, int64_t f,
                                         int32_t *__restrict__ out,
                                         int64_t out_pitch, int32_t *err) {
  const int64_t total = nrows * m;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
       idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / m, j = idx - r * m;
    const int32_t *p = in + r * in_pitch + j * f;
    int64_t s = 0;
    for (int64_t i = 0; i < f; ++i) s += p[i];
    if (s < INT32_MIN || s > INT32_MAX) atomicExch(err, kErrRange);
    out[r * out_pitch + j] = (int32_t)s;
  }
}

__global__ void downsample_warp_kernel(const int32_t *__restrict__ in,
                                       int64_t nrows, int64_t m,
                                       int64_t in_pitch, int64_t f,
                                       int32_t *__restrict__ out,
                                       int64_t out_pitch, int32_t *err) {
  const int lane = threadIdx.x & 31;
  const int64_t total = nrows * m;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t idx = w0; idx < total; idx += nw) {
    const int64_t r = idx / m, j = idx - r * m;
    const int32_t *p = in + r * in_pitch + j * f;
    long long s = 0;
    for (int64_t i = lane; i < f; i += 32) s += p[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      if (s < INT32_MIN || s > INT32_MAX) atomicExch(err, kErrRange);
      out[r * out_pitch + j] = (int32_t)s;
    }
  }
}

// Shared memory of one de-reddening block for spans of up to ns elements.
struct DrLayout {
  int ns, nw;            // span elements, bit words (+1 zero pad word)
  size_t cur, nxt, bits, pref, total;
  __host__ __device__ DrLayout(int ns_) : ns(ns_) {
    nw = (ns + 31) / 32 + 1;
    cur = 512;     // scratch first: 32 uint32 sums, 2 x 16 int64 extremes
    nxt = cur + (size_t)ns * 4;
    bits = nxt + (size_t)ns * 4;
    pref = bits + (size_t)kDrMaxLevels * nw * 4;
    total = pref + (size_t)kDrMaxLevels * nw * 4;
  }
};

__global__ void __launch_bounds__(kDrThreads)
dered_kernel(const int32_t *__restrict__ in, int64_t n, int64_t in_pitch,
             int64_t h, int T, int32_t *__restrict__ out, int64_t out_pitch,
             int ns_max, int32_t *err) {
  extern __shared__ __align__(16) unsigned char smem[];
  const DrLayout Lay(ns_max);
  uint32_t *red = reinterpret_cast<uint32_t *>(smem);            // [32]
  int64_t *rmin = reinterpret_cast<int64_t *>(smem + 128);       // [16]
  int64_t *rmax = reinterpret_cast<int64_t *>(smem + 256);       // [16]
  uint32_t *cur = reinterpret_cast<uint32_t *>(smem + Lay.cur);
  uint32_t *nxt = reinterpret_cast<uint32_t *>(smem + Lay.nxt);
  uint32_t *bits = reinterpret_cast<uint32_t *>(smem + Lay.bits);
  uint32_t *pref = reinterpret_cast<uint32_t *>(smem + Lay.pref);
  __shared__ uint32_t zeros[kDrMaxLevels];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = blockDim.x >> 5;
  const int64_t row = blockIdx.y;
  const int64_t t0 = (int64_t)blockIdx.x * T;
  const int64_t s0 = max((int64_t)0, t0 - h);
  const int64_t s1 = min(n, t0 + T + h);
  const int ns = (int)(s1 - s0);
  const int nw = (ns + 31) / 32;
  const int32_t *x = in + row * in_pitch;

  // ---- span minimum and maximum
  int32_t mn = INT32_MAX, mx = INT32_MIN;
  for (int i = tid; i < ns; i += blockDim.x) {
    const int32_t v = x[s0 + i];
    mn = min(mn, v);
    mx = max(mx, v);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if (lane == 0) {
    rmin[warp] = mn;
    rmax[warp] = mx;
  }
  __syncthreads();
  if (tid == 0) {
    int64_t a = INT64_MAX, b = INT64_MIN;
    for (int w = 0; w < nwarps; ++w) {
      a = min(a, rmin[w]);
      b = max(b, rmax[w]);
    }
    rmin[0] = a;
    rmax[0] = b;
  }
  __syncthreads();
  const int32_t vmin = (int32_t)rmin[0];
  const uint32_t range = (uint32_t)(rmax[0] - rmin[0]);
  const int L = range == 0 ? 0 : 32 - __clz(range);
  __syncthreads();
  for (int i = tid; i < ns; i += blockDim.x)
    cur[i] = (uint32_t)((int64_t)x[s0 + i] - (int64_t)vmin);
  __syncthreads();

  // ---- wavelet matrix, MSB first
  for (int lev = 0; lev < L; ++lev) {
    const int b = L - 1 - lev;
    uint32_t *bw = bits + (size_t)lev * Lay.nw;
    uint32_t *pw = pref + (size_t)lev * Lay.nw;
    for (int w = warp; w <= nw; w += nwarps) {
      const int i = w * 32 + lane;
      const uint32_t bit = i < ns ? (cur[i] >> b) & 1u : 0u;
      const uint32_t word = __ballot_sync(0xffffffffu, bit);
      if (lane == 0) bw[w] = word;
    }
    __syncthreads();
    // exclusive prefix of the words' popcounts (nw + 1 <= blockDim.x)
    {
      const uint32_t c = tid <= nw ? __popc(bw[tid]) : 0u;
      uint32_t inc = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
      }
      if (lane == 31) red[warp] = inc;
      __syncthreads();
      uint32_t below = 0;
      for (int w = 0; w < warp; ++w) below += red[w];
      if (tid <= nw) pw[tid] = below + inc - c;
      if (tid == 0) {
        uint32_t ones = 0;
        for (int w = 0; w < nwarps; ++w) ones += red[w];
        zeros[lev] = (uint32_t)ns - ones;
      }
    }
    __syncthreads();
    const uint32_t Z = zeros[lev];
    for (int i = tid; i < ns; i += blockDim.x) {
      const uint32_t v = cur[i];
      const uint32_t word = bw[i >> 5];
      const uint32_t r1 = pw[i >> 5] + __popc(word & ((1u << (i & 31)) - 1u));
      const uint32_t pos = ((v >> b) & 1u) ? Z + r1 : (uint32_t)i - r1;
      nxt[pos] = v;
    }
    __syncthreads();
    uint32_t *t = cur;
    cur = nxt;
    nxt = t;
  }

  // ---- one k-th-smallest query per output
  const int64_t tend = min(n, t0 + T);
  for (int64_t t = t0 + tid; t < tend; t += blockDim.x) {
    const int64_t a = max((int64_t)0, t - h), bb = min(n - 1, t + h);
    uint32_t l = (uint32_t)(a - s0), r = (uint32_t)(bb - s0 + 1);
    uint32_t k = (r - l - 1) / 2;
    uint32_t res = 0;
    for (int lev = 0; lev < L; ++lev) {
      const uint32_t *bw = bits + (size_t)lev * Lay.nw;
      const uint32_t *pw = pref + (size_t)lev * Lay.nw;
      const uint32_t ol = pw[l >> 5] + __popc(bw[l >> 5] & ((1u << (l & 31)) - 1u));
      const uint32_t orr = pw[r >> 5] + __popc(bw[r >> 5] & ((1u << (r & 31)) - 1u));
      const uint32_t zl = l - ol, zr = r - orr;
      if (k < zr - zl) {
        l = zl;
        r = zr;
      } else {
        k -= zr - zl;
        l = zeros[lev] + ol;
        r = zeros[lev] + orr;
        res |= 1u << (L - 1 - lev);
      }
    }
    const int64_t zv = (int64_t)x[t] - ((int64_t)vmin + (int64_t)res);
    if (zv < INT32_MIN || zv > INT32_MAX) atomicExch(err, kErrRange);
    out[row * out_pitch + t] = (int32_t)zv;
  }
}

}  // namespace

// Outputs per de-reddening block for half-window h: the largest T in
// 8192 .. 512 whose span layout keeps two blocks per SM (else one); 0 if
// even T = 512 does not fit.
int dered_chunk(int64_t h, size_t *smem) {
  for (size_t budget : {kSmemBudgetTwoBlocks, kSmemBudgetOneBlock}) {
    for (int T = 8192; T >= 512; T /= 2) {
      const int64_t ns = T + 2 * h;
      if (ns > (int64_t)kDrThreads * 32 - 32) continue;   // one prefix scan
      const DrLayout L((int)ns);
      if (L.total <= budget) {
        *smem = L.total;
        return T;
      }
    }
  }
  return 0;
}

cudaError_t launch_downsample(const int32_t *d_in, int64_t nrows, int64_t n,
                              int64_t in_pitch, int64_t f, int32_t *d_out,
                              int64_t out_pitch, int32_t *d_err,
                              cudaStream_t s) {
  const int64_t m = n / f;
  if (m <= 0 || nrows <= 0) return cudaSuccess;
  const int64_t total = nrows * m;
  if (f < 32) {
    const int64_t blocks = std::min<int64_t>((total + kDsThreads - 1) / kDsThreads,
                                             148 * 16);
    downsample_thread_kernel<<<(unsigned)blocks, kDsThreads, 0, s>>>(
        d_in, nrows, m, in_pitch, f, d_out, out_pitch, d_err);
  } else {
    const int64_t blocks = std::min<int64_t>((total + 7) / 8, 148 * 16);
    downsample_warp_kernel<<<(unsigned)blocks, kDsThreads, 0, s>>>(
        d_in, nrows, m, in_pitch, f, d_out, out_pitch, d_err);
  }
  return cudaGetLastError();
}

cudaError_t launch_dered(const int32_t *d_in, int64_t nrows, int64_t n,
                         int64_t in_pitch, int64_t h, int32_t *d_out,
                         int64_t out_pitch, int32_t *d_err, cudaStream_t s) {
  size_t smem = 0;
  const int T = dered_chunk(h, &smem);
  if (T == 0) return cudaErrorInvalidValue;
  {
    cudaError_t e = smem_opt_in(dered_kernel);
    if (e != cudaSuccess) return e;
  }
  const int ns_max = (int)std::min<int64_t>(n, T + 2 * h);
  dim3 grid((unsigned)((n + T - 1) / T), (unsigned)nrows);
  dered_kernel<<<grid, kDrThreads, smem, s>>>(d_in, n, in_pitch, h, T, d_out,
                                              out_pitch, ns_max, d_err);
  return cudaGetLastError();
}

}  // namespace ddsp

using namespace ddsp;

extern "C" int ddsp_downsample(ddsp_plan *h, const int32_t *d_in, int64_t nrows,
                               int64_t nsamp, int64_t in_pitch, int64_t factor,
                               int32_t *d_out, int64_t out_pitch,
                               ddsp_stream_t stream) {
  if (!h || !d_in || nrows <= 0 || nsamp <= 0 || factor < 1 ||
      in_pitch < nsamp || out_pitch < nsamp / factor)
    return DDSP_E_INVALID_ARG;
  if (nsamp / factor == 0) return DDSP_OK;        // no complete group
  if (!d_out) return DDSP_E_INVALID_ARG;
  DeviceGuard g(h->p.device);
  return cuda_rc(launch_downsample(d_in, nrows, nsamp, in_pitch, factor, d_out,
                                   out_pitch, h->p.d_err,
                                   reinterpret_cast<cudaStream_t>(stream)));
}

extern "C" int ddsp_dered(ddsp_plan *h, const int32_t *d_in, int64_t nrows,
                          int64_t nsamp, int64_t in_pitch, int64_t half_window,
                          int32_t *d_out, int64_t out_pitch,
                          ddsp_stream_t stream) {
  size_t smem = 0;
  if (!h || !d_in || !d_out || nrows <= 0 || nrows > 65535 || nsamp <= 0 ||
      half_window < 0 || in_pitch < nsamp || out_pitch < nsamp ||
      dered_chunk(half_window, &smem) == 0 || nsamp >= ((int64_t)1 << 31))
    return DDSP_E_INVALID_ARG;
  if (d_in == d_out) return DDSP_E_INVALID_ARG;   // blocks read others' spans
  DeviceGuard g(h->p.device);
  return cuda_rc(launch_dered(d_in, nrows, nsamp, in_pitch, half_window, d_out,
                              out_pitch, h->p.d_err,
                              reinterpret_cast<cudaStream_t>(stream)));
}
