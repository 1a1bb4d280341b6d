// k_rfi.cu -- gptool-style RFI mitigation of a block of 8-bit spectra
// (Sec.2.1: bandpass from the mean spectrum median-filtered over 21
// channels, channels beyond 4 sigma of the corrected mean spectrum and time
// samples beyond 3 sigma of the frequency-averaged series flagged, both done
// twice).  Every step is exact integer arithmetic:
//   s[c] = sum over unflagged t of x[t][c];  b[c] = lower median of s over
//   [c - hw, c + hw] clamped;  R = lower median of b;  e[c] = round(s R / b);
//   channels with 20000 |2e - m2| > kc 14826 mad4 among the unflagged ones
//   ((m2, mad4) = 2 median, 4 MAD of e) are flagged;  y = min(255,
//   round(x R / b));  u[t] = sum of y over unflagged channels;  samples
//   with 20000 |2u - m2| > kt 14826 mad4 are flagged;  after the rounds
//   flagged channels and samples get min(255, round(R / T')).
//
// Per round: channel sums (a channel-group x row-chunk grid, int64
// atomics), one block for the channel statistics (moving medians by
// counting, exact order statistics by histogram narrowing on int64 keys,
// flags, and a 256-entry table y(x) per channel), the time sums (one block
// per row through the tables), one block for the time statistics; then one
// pass writes the block.  One block per statistics step: a few thousand to
// a few hundred thousand values, each pass a coalesced read.
#include <limits.h>
#include <stdint.h>

#include <algorithm>
#include <new>

#include "host.h"

namespace ddsp {
namespace {

constexpr int kRfiThreads = 1024;
constexpr int kRfiBins = 2048;
constexpr int kRfiMaxChan = 8192;
constexpr int kRfiMaxHalf = 32;
constexpr long long kRfiMaxSamples = 1ll << 22;   // s * R stays below 2^63
constexpr int kRfiMaxSigma = 100;

struct RfiState {
  long long R, fill, tkeep;
  int round;
  int pad;
};

struct RfiShared {
  unsigned int hist[kRfiBins];
  unsigned int wsum[kRfiThreads / 32];
  long long red[kRfiThreads / 32][2];
  long long bc[4];
};

__device__ __forceinline__ long long round_div(long long a, long long b) {
  return (2 * a + b) / (2 * b);
}

// Block-wide min and max of the included keys.
template <typename Key>
__device__ void block_minmax(Key key, long long n, RfiShared &sh,
                             long long &mn, long long &mx, long long &cnt) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long a = LLONG_MAX, b = LLONG_MIN, c = 0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    long long v;
    if (key(i, v)) {
      a = min(a, v);
      b = max(b, v);
      ++c;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = min(a, (long long)__shfl_xor_sync(0xffffffffu, a, o));
    b = max(b, (long long)__shfl_xor_sync(0xffffffffu, b, o));
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  __syncthreads();
  if (lane == 0) {
    sh.red[warp][0] = a;
    sh.red[warp][1] = b;
    sh.bc[3] = 0;
  }
  __syncthreads();
  if (lane == 0) atomicAdd((unsigned long long *)&sh.bc[3], (unsigned long long)c);
  __syncthreads();
  if (threadIdx.x == 0) {
    long long x = LLONG_MAX, y = LLONG_MIN;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      x = min(x, sh.red[w][0]);
      y = max(y, sh.red[w][1]);
    }
    sh.bc[0] = x;
    sh.bc[1] = y;
  }
  __syncthreads();
  mn = sh.bc[0];
  mx = sh.bc[1];
  cnt = sh.bc[3];
  __syncthreads();
}

// The k-th smallest (0-based) included key, k < count, keys in [mn, mx]:
// a 2048-bin histogram over the current key range narrows it by 2^11 per
// pass until a bin is one key wide.
template <typename Key>
__device__ long long block_select(Key key, long long n, long long k,
                                  long long mn, long long mx, RfiShared &sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = blockDim.x >> 5;
  long long lo = mn;
  unsigned long long span = (unsigned long long)(mx - mn) + 1ull;
  long long below = 0;
  while (true) {
    int s = 0;
    while (((span - 1ull) >> s) >= (unsigned long long)kRfiBins) ++s;
    const int nb = (int)((span - 1ull) >> s) + 1;
    for (int i = tid; i < nb; i += blockDim.x) sh.hist[i] = 0;
    __syncthreads();
    for (long long i = tid; i < n; i += blockDim.x) {
      long long v;
      if (key(i, v)) {
        const unsigned long long d = (unsigned long long)(v - lo);
        if (v >= lo && d < span) atomicAdd(&sh.hist[d >> s], 1u);
      }
    }
    __syncthreads();
    // exclusive scan over the bins, two per thread (nb <= 2048)
    unsigned int c0 = 2 * tid < nb ? sh.hist[2 * tid] : 0u;
    unsigned int c1 = 2 * tid + 1 < nb ? sh.hist[2 * tid + 1] : 0u;
    unsigned int inc = c0 + c1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int u = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += u;
    }
    if (lane == 31) sh.wsum[warp] = inc;
    __syncthreads();
    unsigned int before = 0;
    for (int w = 0; w < warp; ++w) before += sh.wsum[w];
    const long long run0 = below + (long long)(before + inc - c0 - c1);
    const long long want = k;
    if (2 * tid < nb && run0 <= want && want < run0 + c0) {
      sh.bc[0] = 2 * tid;
      sh.bc[1] = run0;
    }
    if (2 * tid + 1 < nb && run0 + c0 <= want && want < run0 + c0 + c1) {
      sh.bc[0] = 2 * tid + 1;
      sh.bc[1] = run0 + c0;
    }
    __syncthreads();
    const long long bsel = sh.bc[0], bbelow = sh.bc[1];
    __syncthreads();
    (void)nwarps;
    if (s == 0) return lo + bsel;
    lo += bsel << s;
    below = bbelow;
    const unsigned long long rest = span - ((unsigned long long)bsel << s);
    span = min(1ull << s, rest);
  }
}

// (2 median, 4 MAD) of the included keys (count >= 1), like the search's
// window statistics: two middle order statistics, then those of |2v - m2|.
template <typename Key>
__device__ void block_median_mad(Key key, long long n, RfiShared &sh,
                                 long long &m2, long long &mad4,
                                 long long &cnt) {
  long long mn, mx;
  block_minmax(key, n, sh, mn, mx, cnt);
  if (cnt == 0) {
    m2 = mad4 = 0;
    return;
  }
  const long long a = block_select(key, n, (cnt - 1) / 2, mn, mx, sh);
  const long long b = block_select(key, n, cnt / 2, mn, mx, sh);
  m2 = a + b;
  const long long med2 = m2;
  auto dev = [&](long long i, long long &v) {
    long long x;
    if (!key(i, x)) return false;
    const long long d = 2 * x - med2;
    v = d < 0 ? -d : d;
    return true;
  };
  long long dmn, dmx, dc;
  block_minmax(dev, n, sh, dmn, dmx, dc);
  const long long c = block_select(dev, n, (cnt - 1) / 2, dmn, dmx, sh);
  const long long d = block_select(dev, n, cnt / 2, dmn, dmx, sh);
  mad4 = c + d;
}

// ---- per round: channel sums over unflagged samples (four channels per
// thread with 32-bit loads when the row length allows it)
__global__ void rfi_chan_sum(const uint8_t *__restrict__ x, long long nt, int nc,
                             const uint8_t *__restrict__ ft, int rows_per_block,
                             bool vec, unsigned long long *s) {
  const long long t0 = (long long)blockIdx.y * rows_per_block;
  const long long t1 = min(nt, t0 + rows_per_block);
  if (vec) {                  // rows of a multiple of 4 bytes, 4-byte aligned
    const int c4 = blockIdx.x * blockDim.x + threadIdx.x;
    if (4 * c4 >= nc) return;
    unsigned int a0 = 0, a1 = 0, a2 = 0, a3 = 0;   // <= 255 * rows_per_block
    for (long long t = t0; t < t1; ++t) {
      if (ft[t]) continue;
      const uint32_t w = *reinterpret_cast<const uint32_t *>(x + t * nc + 4 * c4);
      a0 += w & 0xFF;
      a1 += (w >> 8) & 0xFF;
      a2 += (w >> 16) & 0xFF;
      a3 += w >> 24;
    }
    if (a0) atomicAdd(&s[4 * c4], (unsigned long long)a0);
    if (a1) atomicAdd(&s[4 * c4 + 1], (unsigned long long)a1);
    if (a2) atomicAdd(&s[4 * c4 + 2], (unsigned long long)a2);
    if (a3) atomicAdd(&s[4 * c4 + 3], (unsigned long long)a3);
    return;
  }
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  unsigned long long acc = 0;
  for (long long t = t0; t < t1; ++t)
    if (!ft[t]) acc += x[t * nc + c];
  if (acc) atomicAdd(&s[c], acc);
}

// ---- per round: channel statistics, flags and the tables (one block)
__global__ void __launch_bounds__(kRfiThreads)
rfi_chan_stats(const unsigned long long *__restrict__ s_in, int nc, int hw,
               int kc, const uint8_t *__restrict__ ft, long long nt,
               long long *b_out, uint8_t *fc, uint8_t *lut, RfiState *st) {
  __shared__ RfiShared sh;
  extern __shared__ long long dyn[];        // sums, then bandpass: 2 nc
  long long *sv = dyn, *bv = dyn + nc;
  for (int c = threadIdx.x; c < nc; c += blockDim.x) sv[c] = (long long)s_in[c];
  __syncthreads();
  // bandpass: lower median of the clamped window, by counting
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    const int lo = max(0, c - hw), hi = min(nc - 1, c + hw);
    const int m = hi - lo + 1, k = (m - 1) / 2;
    long long med = sv[lo];
    for (int j = lo; j <= hi; ++j) {
      const long long v = sv[j];
      int less = 0, leq = 0;
      for (int i = lo; i <= hi; ++i) {
        less += sv[i] < v;
        leq += sv[i] <= v;
      }
      if (less <= k && k < leq) {
        med = v;
        break;
      }
    }
    bv[c] = med;
    b_out[c] = med;
  }
  __syncthreads();
  // reference level R: lower median of the bandpass
  auto bkey = [&](long long i, long long &v) {
    v = bv[i];
    return true;
  };
  long long mn, mx, cnt;
  block_minmax(bkey, nc, sh, mn, mx, cnt);
  const long long R = block_select(bkey, nc, (nc - 1) / 2, mn, mx, sh);
  // corrected channel sums (in place of the sums) and the channel flags
  for (int c = threadIdx.x; c < nc; c += blockDim.x)
    sv[c] = bv[c] > 0 ? round_div(sv[c] * R, bv[c]) : 0;
  __syncthreads();
  auto ekey = [&](long long i, long long &v) {
    if (fc[i]) return false;
    v = sv[i];
    return true;
  };
  long long m2, mad4, ne;
  block_median_mad(ekey, nc, sh, m2, mad4, ne);
  __syncthreads();
  if (ne > 0 && mad4 > 0) {
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
      if (fc[c]) continue;
      const long long d = 2 * sv[c] - m2;
      if (20000 * (d < 0 ? -d : d) > (long long)kc * 14826 * mad4) fc[c] = 1;
    }
  }
  // unflagged samples of this round and the fill level
  unsigned long long kept = 0;
  for (long long t = threadIdx.x; t < nt; t += blockDim.x) kept += !ft[t];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, o);
  __syncthreads();
  if (threadIdx.x == 0) sh.bc[2] = 0;
  __syncthreads();
  if ((threadIdx.x & 31) == 0)
    atomicAdd((unsigned long long *)&sh.bc[2], kept);
  __syncthreads();
  if (threadIdx.x == 0) {
    const long long tk = sh.bc[2];
    st->R = R;
    st->tkeep = tk;
    st->fill = tk > 0 ? min(round_div(R, tk), 255ll) : 0;
  }
}

// ---- per round: the tables y(x) = min(255, round(x R / b)) per channel
__global__ void rfi_tables(const long long *__restrict__ b, int nc,
                           const RfiState *st, uint8_t *lut) {
  const long long R = st->R;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
       i < (long long)nc * 256; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i >> 8), xv = (int)(i & 255);
    const long long bc = b[c];
    const long long y = bc > 0 ? round_div((long long)xv * R, bc) : 0;
    lut[i] = (uint8_t)min(y, 255ll);
  }
}

// ---- per round: the frequency-averaged series through the tables, one
// block per row (grid-stride), threads along the row
__global__ void rfi_time_sum(const uint8_t *__restrict__ x, long long nt, int nc,
                             const uint8_t *__restrict__ fc,
                             const uint8_t *__restrict__ lut, long long *u) {
  __shared__ unsigned long long ws[32];
  for (long long t = blockIdx.x; t < nt; t += gridDim.x) {
    unsigned long long acc = 0;
    const uint8_t *row = x + t * nc;
    for (int c = threadIdx.x; c < nc; c += blockDim.x)
      if (!fc[c]) acc += lut[(long long)c * 256 + row[c]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long tot = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += ws[w];
      u[t] = (long long)tot;
    }
    __syncthreads();
  }
}

// ---- per round: time statistics and flags (one block)
__global__ void __launch_bounds__(kRfiThreads)
rfi_time_stats(const long long *__restrict__ u, long long nt, int kt,
               uint8_t *ft) {
  __shared__ RfiShared sh;
  auto ukey = [&](long long i, long long &v) {
    if (ft[i]) return false;
    v = u[i];
    return true;
  };
  long long m2, mad4, n;
  block_median_mad(ukey, nt, sh, m2, mad4, n);
  __syncthreads();
  if (n == 0 || mad4 <= 0) return;
  for (long long t = threadIdx.x; t < nt; t += blockDim.x) {
    if (ft[t]) continue;
    const long long d = 2 * u[t] - m2;
    if (20000 * (d < 0 ? -d : d) > (long long)kt * 14826 * mad4) ft[t] = 1;
  }
}

// ---- the cleaned block, one block per row (grid-stride), 32-bit accesses
// when the rows allow them
__global__ void rfi_apply(const uint8_t *__restrict__ x, long long nt, int nc,
                          const uint8_t *__restrict__ fc,
                          const uint8_t *__restrict__ ft,
                          const uint8_t *__restrict__ lut, const RfiState *st,
                          bool vec, uint8_t *out) {
  const uint8_t fill = (uint8_t)st->fill;
  for (long long t = blockIdx.x; t < nt; t += gridDim.x) {
    const uint8_t *xr = x + t * nc;
    uint8_t *orow = out + t * nc;
    if (ft[t]) {
      for (int c = threadIdx.x; c < nc; c += blockDim.x) orow[c] = fill;
      continue;
    }
    if (vec) {
      for (int c4 = threadIdx.x; 4 * c4 < nc; c4 += blockDim.x) {
        const uint32_t w = reinterpret_cast<const uint32_t *>(xr)[c4];
        uint32_t o = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int c = 4 * c4 + q;
          const uint32_t v = (w >> (8 * q)) & 0xFF;
          const uint32_t y = fc[c] ? fill : lut[(long long)c * 256 + v];
          o |= y << (8 * q);
        }
        reinterpret_cast<uint32_t *>(orow)[c4] = o;
      }
    } else {
      for (int c = threadIdx.x; c < nc; c += blockDim.x)
        orow[c] = fc[c] ? fill : lut[(long long)c * 256 + xr[c]];
    }
  }
}

}  // namespace
}  // namespace ddsp

using namespace ddsp;

struct ddsp_rfi {
  int device = 0;
  long long max_nt = 0;
  int max_nc = 0;
  unsigned long long *s = nullptr;
  long long *b = nullptr, *u = nullptr;
  uint8_t *fc = nullptr, *ft = nullptr, *lut = nullptr;
  RfiState *st = nullptr;
  long long nt = 0;
  int nc = 0;
  cudaStream_t last = nullptr;
  bool ran = false;
};

static void rfi_free(ddsp_rfi *r) {
  void *p[] = {r->s, r->b, r->u, r->fc, r->ft, r->lut, r->st};
  for (void *q : p) cudaFree(q);
}

extern "C" int ddsp_rfi_create(ddsp_rfi **out, int device, int64_t max_nsamp,
                               int max_nchan) {
  if (!out || max_nsamp < 1 || max_nsamp > kRfiMaxSamples || max_nchan < 1 ||
      max_nchan > kRfiMaxChan)
    return DDSP_E_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return DDSP_E_INVALID_ARG;
  DeviceGuard g(device);
  ddsp_rfi *r = new (std::nothrow) ddsp_rfi;
  if (!r) return DDSP_E_NOMEM;
  r->device = device;
  r->max_nt = max_nsamp;
  r->max_nc = max_nchan;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void **p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  alloc((void **)&r->s, (size_t)max_nchan * 8);
  alloc((void **)&r->b, (size_t)max_nchan * 8);
  alloc((void **)&r->u, (size_t)max_nsamp * 8);
  alloc((void **)&r->fc, (size_t)max_nchan);
  alloc((void **)&r->ft, (size_t)max_nsamp);
  alloc((void **)&r->lut, (size_t)max_nchan * 256);
  alloc((void **)&r->st, sizeof(RfiState));
  if (e != cudaSuccess) {
    rfi_free(r);
    delete r;
    return cuda_rc(e);
  }
  *out = r;
  return DDSP_OK;
}

extern "C" void ddsp_rfi_destroy(ddsp_rfi *r) {
  if (!r) return;
  DeviceGuard g(r->device);
  cudaDeviceSynchronize();
  rfi_free(r);
  delete r;
}

extern "C" int ddsp_rfi_clean(ddsp_rfi *r, const uint8_t *d_in, int64_t nsamp,
                              int nchan, int half_window, int kc, int kt,
                              int rounds, uint8_t *d_out,
                              ddsp_stream_t stream) {
  if (!r || !d_in || !d_out || nsamp < 1 || nsamp > r->max_nt || nchan < 1 ||
      nchan > r->max_nc || half_window < 0 || half_window > kRfiMaxHalf ||
      kc < 0 || kt < 0 || kc > kRfiMaxSigma || kt > kRfiMaxSigma ||
      rounds < 1 || rounds > 16)
    return DDSP_E_INVALID_ARG;
  DeviceGuard g(r->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t csmem = (size_t)2 * nchan * 8;
  cudaError_t ea = smem_opt_in(rfi_chan_stats);
  if (ea != cudaSuccess) return cuda_rc(ea);
  cudaError_t e = cudaMemsetAsync(r->fc, 0, (size_t)nchan, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(r->ft, 0, (size_t)nsamp, s);
  if (e != cudaSuccess) return cuda_rc(e);
  const int rows = 256;
  // 32-bit accesses only for rows of whole words at word-aligned addresses
  const bool vec = (nchan & 3) == 0 &&
                   (reinterpret_cast<uintptr_t>(d_in) & 3) == 0 &&
                   (reinterpret_cast<uintptr_t>(d_out) & 3) == 0;
  const int cols = vec ? nchan / 4 : nchan;
  dim3 gsum((unsigned)((cols + 255) / 256), (unsigned)((nsamp + rows - 1) / rows));
  const unsigned glut = (unsigned)std::min<long long>(((long long)nchan * 256 + 255) / 256, 148 * 8);
  const unsigned grows = (unsigned)std::min<int64_t>(nsamp, 148 * 8);
  for (int rd = 0; rd < rounds; ++rd) {
    e = cudaMemsetAsync(r->s, 0, (size_t)nchan * 8, s);
    if (e != cudaSuccess) return cuda_rc(e);
    rfi_chan_sum<<<gsum, 256, 0, s>>>(d_in, nsamp, nchan, r->ft, rows, vec, r->s);
    rfi_chan_stats<<<1, kRfiThreads, csmem, s>>>(r->s, nchan, half_window, kc,
                                             r->ft, nsamp, r->b, r->fc, r->lut,
                                             r->st);
    rfi_tables<<<glut, 256, 0, s>>>(r->b, nchan, r->st, r->lut);
    rfi_time_sum<<<grows, 256, 0, s>>>(d_in, nsamp, nchan, r->fc, r->lut, r->u);
    rfi_time_stats<<<1, kRfiThreads, 0, s>>>(r->u, nsamp, kt, r->ft);
  }
  rfi_apply<<<grows, 256, 0, s>>>(d_in, nsamp, nchan, r->fc, r->ft, r->lut,
                                  r->st, vec, d_out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_rc(e);
  r->nt = nsamp;
  r->nc = nchan;
  r->last = s;
  r->ran = true;
  return DDSP_OK;
}

extern "C" int ddsp_rfi_flags(ddsp_rfi *r, uint8_t *host_chan_flags,
                              uint8_t *host_time_flags, int64_t *fill) {
  if (!r) return DDSP_E_INVALID_ARG;
  if (!r->ran) return DDSP_E_STATE;
  DeviceGuard g(r->device);
  cudaError_t e = cudaStreamSynchronize(r->last);
  if (e == cudaSuccess && host_chan_flags)
    e = cudaMemcpy(host_chan_flags, r->fc, (size_t)r->nc, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && host_time_flags)
    e = cudaMemcpy(host_time_flags, r->ft, (size_t)r->nt, cudaMemcpyDeviceToHost);
  RfiState st{};
  if (e == cudaSuccess) e = cudaMemcpy(&st, r->st, sizeof st, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_rc(e);
  if (fill) *fill = st.fill;
  return DDSP_OK;
}
