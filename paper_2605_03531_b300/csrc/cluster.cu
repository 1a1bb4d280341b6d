// cluster.cu -- peaks filtering and DM-time clustering of single-pulse
// candidates (Sec.2.1: redundant candidates of one event are removed with
// square stencils in the DM-time plane, the rest are clustered with DBSCAN
// and the strongest candidate of each cluster is kept).
//
// Data layout: the candidates of one call mark bits in a plane bitmap
// (ndm rows of ceil(nsamp/32) words, plus one zero pad word), and an
// exclusive prefix sum of the words' popcounts gives every set bit its rank.
// The rank of (k, t) is the record's position in (dm_idx, t) order, so one
// scatter sorts the records, and the number of candidates of row k between
// two times is a difference of two ranks: every stencil or neighbourhood
// query reads only the rows it covers.  The peaks get a bitmap of their own.
//
//   1. mark the candidates (out-of-plane records, bad width indices and
//      repeated (dm_idx, t) set an error word), prefix-sum, scatter sorted;
//   2. peaks: a candidate stays unless a stronger one (larger S/N, ties to
//      the earlier (dm_idx, t)) lies in its square stencil of half-size
//      half[w_idx]; rows are scanned nearest first and the scan stops at the
//      first stronger record: one thread per candidate takes the rows within
//      distance 2 (most candidates end there), and the few still undecided
//      are queued for one warp each, 32 rows at a time, so a wide stencil
//      does not hold a block for hundreds of serial row lookups; survivors
//      mark the peak bitmap;
//   3. DBSCAN on the sorted peaks: neighbour counts from ranks (core if
//      >= min_pts), a lock-free union-find over core-core neighbour pairs
//      that always hooks the larger root under the smaller (so each
//      cluster's root is its smallest core index, the canonical label),
//      border points take the smallest label among their core neighbours;
//   4. representatives: per label the strongest member by an atomicMax on
//      (order-preserving S/N bits << 32 | ~index), compacted in label order
//      through a bitmap of the cluster roots.
// Every retry loop is bounded and reports through the error word.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "host.h"

namespace ddsp {
namespace {

constexpr int kMaxClusterWidths = 32;
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;
constexpr int kScanTile = kScanThreads * kScanPer;   // words per scan block
constexpr uint32_t kErrRecord = 1;      // out of plane or bad width index
constexpr uint32_t kErrRepeat = 2;      // a repeated (dm_idx, t)
constexpr uint32_t kErrLimit = 4;       // a bounded retry loop gave up
constexpr int kUnionLimit = 1 << 24;

struct ClState {
  uint32_t n_in;      // records used this call
  uint32_t err;
  uint32_t n_queue;   // candidates left to the warp-wide stencil scan
  uint32_t pad;
};

// rows of a stencil a thread checks on its own, nearest first (distance
// <= kQuickRows); the candidates still undecided after them are queued for
// a warp that scans 32 rows at a time
constexpr int kQuickRows = 2;

struct HalfTable {
  int32_t h[kMaxClusterWidths];
};

struct Plane {
  const uint32_t *bm;   // bitmap words (nwords + 1, last one zero)
  const uint32_t *pf;   // exclusive popcount prefix (nwords + 1)
  const uint32_t *wmax; // largest ordered S/N key of each word's records
  int64_t wpr;          // words per row
  int ndm;
  int64_t nsamp;
  // rank of (k, tt), 0 <= tt <= nsamp: set bits before it in (k, t) order
  __device__ __forceinline__ uint32_t rank(int k, int64_t tt) const {
    const int64_t w = (int64_t)k * wpr + (tt >> 5);
    const uint32_t b = (uint32_t)(tt & 31);
    return pf[w] + __popc(bm[w] & ((1u << b) - 1u));
  }
  __device__ __forceinline__ uint32_t total() const { return pf[(int64_t)ndm * wpr]; }
};

__device__ __forceinline__ bool stronger(const ddsp_cand &o,
                                         const ddsp_cand &r) {
  if (o.snr != r.snr) return o.snr > r.snr;
  return o.dm_idx < r.dm_idx || (o.dm_idx == r.dm_idx && o.t < r.t);
}

// uint32 whose unsigned order is the float order (finite values; -0 and
// +0 map to one key, as they compare equal)
__device__ __forceinline__ uint32_t ordered_bits(float f) {
  const uint32_t u = __float_as_uint(f == 0.0f ? 0.0f : f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void cl_prep(const uint32_t *d_count, int64_t n, ClState *st) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    uint32_t c = (uint32_t)n;
    if (d_count) c = min(*d_count, (uint32_t)n);
    st->n_in = c;
    st->err = 0;
    st->n_queue = 0;
  }
}

__global__ void cl_zero(uint32_t *p, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 0;
}

__global__ void cl_mark(const ddsp_cand *__restrict__ c, ClState *st,
                        uint32_t *bm, int ndm, int64_t nsamp, int64_t wpr,
                        int nw) {
  const uint32_t n = st->n_in;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const ddsp_cand r = c[i];
    if (r.dm_idx >= (uint32_t)ndm || (int64_t)r.t >= nsamp ||
        r.w_idx >= (uint32_t)nw) {
      atomicOr(&st->err, kErrRecord);
      continue;
    }
    const uint32_t bit = 1u << (r.t & 31);
    const uint32_t old =
        atomicOr(&bm[(int64_t)r.dm_idx * wpr + (r.t >> 5)], bit);
    if (old & bit) atomicOr(&st->err, kErrRepeat);
  }
}

// ---- exclusive prefix of popcounts over nwords words: pf[0..nwords]
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *ws,
                                                    uint32_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) ws[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const int nwarp = blockDim.x >> 5;
    uint32_t x = lane < nwarp ? ws[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += u;
    }
    if (lane < nwarp) ws[lane] = x;   // inclusive warp totals
  }
  __syncthreads();
  const uint32_t below = warp > 0 ? ws[warp - 1] : 0u;
  if (total) *total = ws[(blockDim.x >> 5) - 1];
  return below + inc - v;
}

__global__ void __launch_bounds__(kScanThreads)
scan_reduce(const uint32_t *__restrict__ bm, int64_t nwords, uint32_t *bsum) {
  __shared__ uint32_t ws[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanPer;
  uint32_t s = 0;
#pragma unroll
  for (int q = 0; q < kScanPer; ++q)
    if (base + q < nwords) s += __popc(bm[base + q]);
  uint32_t total;
  block_excl_scan(s, ws, &total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads)
scan_top(uint32_t *bsum, int64_t nblocks, uint32_t *grand_total) {
  __shared__ uint32_t ws[32];
  uint32_t carry = 0;
  for (int64_t b0 = 0; b0 < nblocks; b0 += kScanThreads) {
    const int64_t b = b0 + threadIdx.x;
    const uint32_t v = b < nblocks ? bsum[b] : 0u;
    uint32_t total;
    const uint32_t ex = block_excl_scan(v, ws, &total);
    if (b < nblocks) bsum[b] = carry + ex;
    carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) *grand_total = carry;
}

__global__ void __launch_bounds__(kScanThreads)
scan_down(const uint32_t *__restrict__ bm, int64_t nwords,
          const uint32_t *__restrict__ bsum, uint32_t *pf) {
  __shared__ uint32_t ws[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanPer;
  uint32_t c[kScanPer], s = 0;
#pragma unroll
  for (int q = 0; q < kScanPer; ++q) {
    c[q] = base + q < nwords ? __popc(bm[base + q]) : 0u;
    s += c[q];
  }
  uint32_t run = bsum[blockIdx.x] + block_excl_scan(s, ws, nullptr);
#pragma unroll
  for (int q = 0; q < kScanPer; ++q) {
    if (base + q < nwords) pf[base + q] = run;
    run += c[q];
  }
}

cudaError_t scan_words(const uint32_t *bm, int64_t nwords, uint32_t *pf,
                       uint32_t *bsum, cudaStream_t s) {
  const int64_t nb = std::max<int64_t>((nwords + kScanTile - 1) / kScanTile, 1);
  scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(bm, nwords, bsum);
  scan_top<<<1, kScanThreads, 0, s>>>(bsum, nb, pf + nwords);
  scan_down<<<(unsigned)nb, kScanThreads, 0, s>>>(bm, nwords, bsum, pf);
  return cudaGetLastError();
}

// ---- sorted scatter: record i goes to the rank of its bit; each bitmap
// word also keeps the largest S/N key of its records
__global__ void cl_scatter(const ddsp_cand *__restrict__ c, const ClState *st,
                           Plane P, int nw, ddsp_cand *sorted,
                           uint32_t *wmax) {
  const uint32_t n = st->n_in;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const ddsp_cand r = c[i];
    if (r.dm_idx >= (uint32_t)P.ndm || (int64_t)r.t >= P.nsamp ||
        r.w_idx >= (uint32_t)nw)
      continue;
    sorted[P.rank((int)r.dm_idx, r.t)] = r;
    atomicMax(&wmax[(int64_t)r.dm_idx * P.wpr + (r.t >> 5)],
              ordered_bits(r.snr));
  }
}

// ---- peaks filter over the sorted records
// Is any record of row kk inside [t0, t1] (other than record i) stronger
// than r?  Words whose largest S/N is below r's hold none and are skipped;
// the records of the others are checked one by one.
__device__ __forceinline__ bool row_has_stronger(
    const ddsp_cand *__restrict__ sorted, const Plane &P, int64_t kk,
    int64_t t0, int64_t t1, int64_t i, const ddsp_cand &r) {
  const uint32_t key = ordered_bits(r.snr);
  const int64_t row = kk * P.wpr;
  const int64_t w0 = row + (t0 >> 5), w1 = row + (t1 >> 5);
  for (int64_t w = w0; w <= w1; ++w) {
    if (P.wmax[w] < key) continue;
    const uint32_t blo = w == w0 ? (uint32_t)(t0 & 31) : 0u;
    const uint32_t bhi = w == w1 ? (uint32_t)(t1 & 31) : 31u;
    const uint32_t word = P.bm[w];
    uint32_t bits = word & ((2u << bhi) - 1u) & ~((1u << blo) - 1u);
    while (bits) {
      const uint32_t b = __ffs(bits) - 1;
      bits &= bits - 1u;
      const uint32_t j = P.pf[w] + __popc(word & ((1u << b) - 1u));
      if (j != (uint32_t)i && stronger(sorted[j], r)) return true;
    }
  }
  return false;
}

// Row of stencil order o (0: the candidate's own row; 2d - 1 and 2d: the
// rows d below and d above), or -1 outside the plane.
__device__ __forceinline__ int64_t stencil_row(int64_t k, int64_t o, int ndm) {
  const int64_t d = (o + 1) >> 1;
  const int64_t kk = (o & 1) ? k - d : k + d;
  return (kk >= 0 && kk < ndm) ? kk : -1;
}

// One thread per candidate: the rows at distance <= kQuickRows.  Decided
// candidates are done (survivors mark the peak bitmap); the rest queue.
__global__ void cl_peaks_near(const ddsp_cand *__restrict__ sorted, Plane P,
                              HalfTable half, uint32_t *bm_peaks,
                              uint32_t *queue, ClState *st) {
  const uint32_t n = P.total();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const ddsp_cand r = sorted[i];
    const int64_t h = half.h[r.w_idx];
    const int64_t t0 = max((int64_t)0, (int64_t)r.t - h);
    const int64_t t1 = min(P.nsamp - 1, (int64_t)r.t + h);
    // rows nearest first, no further than the plane reaches
    const int64_t dmax = min(h, max((int64_t)r.dm_idx,
                                    (int64_t)P.ndm - 1 - (int64_t)r.dm_idx));
    const int64_t onear = 2 * min(dmax, (int64_t)kQuickRows);
    bool beaten = false;
    for (int64_t o = 0; o <= onear && !beaten; ++o) {
      const int64_t kk = stencil_row(r.dm_idx, o, P.ndm);
      if (kk >= 0) beaten = row_has_stronger(sorted, P, kk, t0, t1, i, r);
    }
    if (beaten) continue;
    if (dmax <= kQuickRows) {
      atomicOr(&bm_peaks[(int64_t)r.dm_idx * P.wpr + (r.t >> 5)],
               1u << (r.t & 31));
    } else {
      queue[atomicAdd(&st->n_queue, 1u)] = (uint32_t)i;
    }
  }
}

// One warp per queued candidate: the remaining rows of its stencil, 32 at a
// time (one per lane), until a lane finds a stronger record.
__global__ void cl_peaks_far(const ddsp_cand *__restrict__ sorted, Plane P,
                             HalfTable half, uint32_t *bm_peaks,
                             const uint32_t *__restrict__ queue,
                             const ClState *st) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const uint32_t nq = st->n_queue;
  for (int64_t q = warp; q < nq; q += nwarps) {
    const int64_t i = queue[q];
    const ddsp_cand r = sorted[i];
    const int64_t h = half.h[r.w_idx];
    const int64_t t0 = max((int64_t)0, (int64_t)r.t - h);
    const int64_t t1 = min(P.nsamp - 1, (int64_t)r.t + h);
    const int64_t dmax = min(h, max((int64_t)r.dm_idx,
                                    (int64_t)P.ndm - 1 - (int64_t)r.dm_idx));
    const int64_t oend = 2 * dmax;              // last stencil order
    bool beaten = false;
    for (int64_t o0 = 2 * kQuickRows + 1; o0 <= oend; o0 += 32) {
      const int64_t o = o0 + lane;
      bool mine = false;
      if (o <= oend) {
        const int64_t kk = stencil_row(r.dm_idx, o, P.ndm);
        if (kk >= 0) mine = row_has_stronger(sorted, P, kk, t0, t1, i, r);
      }
      if (__any_sync(0xffffffffu, mine)) {
        beaten = true;
        break;
      }
    }
    if (!beaten && lane == 0)
      atomicOr(&bm_peaks[(int64_t)r.dm_idx * P.wpr + (r.t >> 5)],
               1u << (r.t & 31));
  }
}

__global__ void cl_gather_peaks(const ddsp_cand *__restrict__ sorted,
                                Plane P, Plane PK, ddsp_cand *peaks) {
  const uint32_t n = P.total();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const ddsp_cand r = sorted[i];
    const int64_t w = (int64_t)r.dm_idx * PK.wpr + (r.t >> 5);
    if (PK.bm[w] & (1u << (r.t & 31))) peaks[PK.rank((int)r.dm_idx, r.t)] = r;
  }
}

// ---- DBSCAN over the sorted peaks
struct Eps {
  int dm, t, min_pts;
};

__global__ void cl_core(const ddsp_cand *__restrict__ peaks, Plane PK, Eps e,
                        uint8_t *core, int32_t *parent) {
  const uint32_t n = PK.total();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const ddsp_cand r = peaks[i];
    const int64_t t0 = max((int64_t)0, (int64_t)r.t - e.t);
    const int64_t t1 = min(PK.nsamp - 1, (int64_t)r.t + e.t);
    const int k0 = max(0, (int)r.dm_idx - e.dm);
    const int k1 = min(PK.ndm - 1, (int)r.dm_idx + e.dm);
    int64_t cnt = 0;
    for (int kk = k0; kk <= k1 && cnt < e.min_pts; ++kk)
      cnt += PK.rank(kk, t1 + 1) - PK.rank(kk, t0);
    core[i] = cnt >= e.min_pts;
    parent[i] = (int32_t)i;
  }
}

// root of x; halves the path on the way (every parent stays <= its child,
// so a stale value is still an ancestor).  Parents are read from L2
// (__ldcg): other blocks hook roots there with atomics.
__device__ __forceinline__ int32_t uf_find(int32_t *parent, int32_t x,
                                           uint32_t *err) {
  for (int it = 0; it < kUnionLimit; ++it) {
    const int32_t p = __ldcg(parent + x);
    if (p == x) return x;
    const int32_t g = __ldcg(parent + p);
    if (g != p) parent[x] = g;
    x = p;
  }
  atomicOr(err, kErrLimit);
  return x;
}

__device__ __forceinline__ void uf_union(int32_t *parent, int32_t a, int32_t b,
                                         uint32_t *err) {
  for (int it = 0; it < kUnionLimit; ++it) {
    a = uf_find(parent, a, err);
    b = uf_find(parent, b, err);
    if (a == b) return;
    if (a < b) {
      const int32_t t = a;
      a = b;
      b = t;
    }
    // hook the larger root under the smaller one, if it is still a root
    const int32_t old = atomicCAS(&parent[a], a, b);
    if (old == a) return;
  }
  atomicOr(err, kErrLimit);
}

__global__ void cl_union(const ddsp_cand *__restrict__ peaks, Plane PK,
                         Eps e, const uint8_t *__restrict__ core,
                         int32_t *parent, ClState *st) {
  const uint32_t n = PK.total();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (!core[i]) continue;
    const ddsp_cand r = peaks[i];
    const int64_t t0 = max((int64_t)0, (int64_t)r.t - e.t);
    const int64_t t1 = min(PK.nsamp - 1, (int64_t)r.t + e.t);
    const int k0 = max(0, (int)r.dm_idx - e.dm);
    const int k1 = min(PK.ndm - 1, (int)r.dm_idx + e.dm);
    for (int kk = k0; kk <= k1; ++kk) {
      const uint32_t lo = PK.rank(kk, t0), hi = PK.rank(kk, t1 + 1);
      // every pair once: from its larger index
      for (uint32_t j = lo; j < hi && j < (uint32_t)i; ++j)
        if (core[j]) uf_union(parent, (int32_t)i, (int32_t)j, &st->err);
    }
  }
}

__global__ void cl_label_core(Plane PK, const uint8_t *__restrict__ core,
                              int32_t *parent, int32_t *label, ClState *st) {
  const uint32_t n = PK.total();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    label[i] = core[i] ? uf_find(parent, (int32_t)i, &st->err) : -1;
}

__global__ void cl_label_border(const ddsp_cand *__restrict__ peaks,
                                Plane PK, Eps e,
                                const uint8_t *__restrict__ core,
                                int32_t *label) {
  const uint32_t n = PK.total();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (core[i]) continue;
    const ddsp_cand r = peaks[i];
    const int64_t t0 = max((int64_t)0, (int64_t)r.t - e.t);
    const int64_t t1 = min(PK.nsamp - 1, (int64_t)r.t + e.t);
    const int k0 = max(0, (int)r.dm_idx - e.dm);
    const int k1 = min(PK.ndm - 1, (int)r.dm_idx + e.dm);
    int32_t best = -1;
    for (int kk = k0; kk <= k1; ++kk) {
      const uint32_t lo = PK.rank(kk, t0), hi = PK.rank(kk, t1 + 1);
      for (uint32_t j = lo; j < hi; ++j)
        if (core[j] && (best < 0 || label[j] < best)) best = label[j];
    }
    label[i] = best;
  }
}

__global__ void cl_repkey(const ddsp_cand *__restrict__ peaks, Plane PK,
                          const int32_t *__restrict__ label,
                          unsigned long long *repkey, uint32_t *bm_roots) {
  const uint32_t n = PK.total();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = label[i];
    if (c < 0) continue;
    const unsigned long long key =
        ((unsigned long long)ordered_bits(peaks[i].snr) << 32) |
        (unsigned long long)(0xffffffffu - (uint32_t)i);
    atomicMax(&repkey[c], key);
    if (c == (int32_t)i) atomicOr(&bm_roots[i >> 5], 1u << (i & 31));
  }
}

__global__ void cl_zero_keys(Plane PK, unsigned long long *repkey) {
  const uint32_t n = PK.total();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    repkey[i] = 0ull;
}

__global__ void cl_gather_reps(const ddsp_cand *__restrict__ peaks, Plane PK,
                               const unsigned long long *__restrict__ repkey,
                               const uint32_t *__restrict__ bm_roots,
                               const uint32_t *__restrict__ pf_roots,
                               ddsp_cand *reps, uint32_t *rep_idx) {
  const uint32_t n = PK.total();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t w = bm_roots[i >> 5], bit = 1u << (i & 31);
    if (!(w & bit)) continue;
    const uint32_t pos = pf_roots[i >> 5] + __popc(w & (bit - 1u));
    const uint32_t r = 0xffffffffu - (uint32_t)(repkey[i] & 0xffffffffull);
    reps[pos] = peaks[r];
    rep_idx[pos] = r;
  }
}

}  // namespace
}  // namespace ddsp

using namespace ddsp;

struct ddsp_cluster {
  int device = 0;
  int ndm = 0;
  int64_t nsamp = 0, wpr = 0, nwords = 0, cap = 0, rwords = 0;
  uint32_t *bm_c = nullptr, *pf_c = nullptr, *bm_p = nullptr, *pf_p = nullptr;
  uint32_t *wmax = nullptr;
  uint32_t *bm_r = nullptr, *pf_r = nullptr, *bsum = nullptr;
  ddsp_cand *sorted = nullptr, *peaks = nullptr, *reps = nullptr;
  uint8_t *core = nullptr;
  int32_t *parent = nullptr, *label = nullptr;
  uint32_t *rep_idx = nullptr, *queue = nullptr;
  unsigned long long *repkey = nullptr;
  ClState *st = nullptr;
  cudaStream_t last = nullptr;
  bool ran = false;
};

static void cluster_free(ddsp_cluster *c) {
  void *ptrs[] = {c->bm_c, c->pf_c, c->bm_p, c->pf_p, c->wmax, c->bm_r, c->pf_r,
                  c->bsum, c->sorted, c->peaks, c->reps, c->core, c->parent,
                  c->label, c->rep_idx, c->queue, c->repkey, c->st};
  for (void *p : ptrs) cudaFree(p);
}

extern "C" int ddsp_cluster_create(ddsp_cluster **out, int device, int ndm,
                                   int64_t nsamp, int64_t capacity) {
  if (!out || ndm <= 0 || nsamp <= 0 || capacity <= 0 ||
      capacity >= ((int64_t)1 << 31) || nsamp >= ((int64_t)1 << 32))
    return DDSP_E_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return DDSP_E_INVALID_ARG;
  DeviceGuard g(device);
  ddsp_cluster *c = new (std::nothrow) ddsp_cluster;
  if (!c) return DDSP_E_NOMEM;
  c->device = device;
  c->ndm = ndm;
  c->nsamp = nsamp;
  c->wpr = (nsamp + 31) / 32;
  c->nwords = (int64_t)ndm * c->wpr;
  c->cap = capacity;
  c->rwords = (capacity + 31) / 32;
  const int64_t nb = std::max<int64_t>(
      (std::max(c->nwords, c->rwords) + kScanTile - 1) / kScanTile, 1);
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void **p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  const size_t pw = (size_t)(c->nwords + 1) * 4;
  alloc((void **)&c->bm_c, pw);
  alloc((void **)&c->pf_c, pw);
  alloc((void **)&c->bm_p, pw);
  alloc((void **)&c->pf_p, pw);
  alloc((void **)&c->wmax, pw);
  alloc((void **)&c->bm_r, (size_t)(c->rwords + 1) * 4);
  alloc((void **)&c->pf_r, (size_t)(c->rwords + 1) * 4);
  alloc((void **)&c->bsum, (size_t)nb * 4);
  alloc((void **)&c->sorted, (size_t)capacity * sizeof(ddsp_cand));
  alloc((void **)&c->peaks, (size_t)capacity * sizeof(ddsp_cand));
  alloc((void **)&c->reps, (size_t)capacity * sizeof(ddsp_cand));
  alloc((void **)&c->core, (size_t)capacity);
  alloc((void **)&c->parent, (size_t)capacity * 4);
  alloc((void **)&c->label, (size_t)capacity * 4);
  alloc((void **)&c->rep_idx, (size_t)capacity * 4);
  alloc((void **)&c->queue, (size_t)capacity * 4);
  alloc((void **)&c->repkey, (size_t)capacity * 8);
  alloc((void **)&c->st, sizeof(ClState));
  if (e != cudaSuccess) {
    cluster_free(c);
    delete c;
    return cuda_rc(e);
  }
  *out = c;
  return DDSP_OK;
}

extern "C" void ddsp_cluster_destroy(ddsp_cluster *c) {
  if (!c) return;
  DeviceGuard g(c->device);
  cudaDeviceSynchronize();
  cluster_free(c);
  delete c;
}

extern "C" int ddsp_peaks_cluster(ddsp_cluster *c, const ddsp_cand *d_cands,
                                  const uint32_t *d_count, int64_t n,
                                  const int32_t *half, int nwidths, int eps_dm,
                                  int eps_t, int min_pts,
                                  ddsp_stream_t stream) {
  if (!c || n < 0 || n > c->cap || (n > 0 && !d_cands) || !half ||
      nwidths < 1 || nwidths > kMaxClusterWidths || eps_dm < 0 || eps_t < 0 ||
      min_pts < 1)
    return DDSP_E_INVALID_ARG;
  HalfTable ht{};
  for (int w = 0; w < nwidths; ++w) {
    if (half[w] < 0) return DDSP_E_INVALID_ARG;
    ht.h[w] = half[w];
  }
  DeviceGuard g(c->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t nwp = c->nwords + 1;
  const unsigned gz = 148 * 8;
  const unsigned gc = (unsigned)std::max<int64_t>(
      1, std::min<int64_t>((n + 255) / 256, 148 * 16));
  Plane P{c->bm_c, c->pf_c, c->wmax, c->wpr, c->ndm, c->nsamp};
  Plane PK{c->bm_p, c->pf_p, nullptr, c->wpr, c->ndm, c->nsamp};
  const Eps ep{eps_dm, eps_t, min_pts};
  cl_prep<<<1, 32, 0, s>>>(d_count, n, c->st);
  cl_zero<<<gz, 256, 0, s>>>(c->bm_c, nwp);
  cl_zero<<<gz, 256, 0, s>>>(c->bm_p, nwp);
  cl_zero<<<gz, 256, 0, s>>>(c->wmax, nwp);
  cl_zero<<<gz, 256, 0, s>>>(c->bm_r, c->rwords + 1);
  cl_mark<<<gc, 256, 0, s>>>(d_cands, c->st, c->bm_c, c->ndm, c->nsamp, c->wpr,
                             nwidths);
  cudaError_t e = scan_words(c->bm_c, c->nwords, c->pf_c, c->bsum, s);
  if (e != cudaSuccess) return cuda_rc(e);
  cl_scatter<<<gc, 256, 0, s>>>(d_cands, c->st, P, nwidths, c->sorted,
                                c->wmax);
  cl_peaks_near<<<gc, 256, 0, s>>>(c->sorted, P, ht, c->bm_p, c->queue, c->st);
  cl_peaks_far<<<148 * 8, 256, 0, s>>>(c->sorted, P, ht, c->bm_p, c->queue,
                                       c->st);
  e = scan_words(c->bm_p, c->nwords, c->pf_p, c->bsum, s);
  if (e != cudaSuccess) return cuda_rc(e);
  cl_gather_peaks<<<gc, 256, 0, s>>>(c->sorted, P, PK, c->peaks);
  cl_core<<<gc, 256, 0, s>>>(c->peaks, PK, ep, c->core, c->parent);
  cl_union<<<gc, 256, 0, s>>>(c->peaks, PK, ep, c->core, c->parent, c->st);
  cl_label_core<<<gc, 256, 0, s>>>(PK, c->core, c->parent, c->label, c->st);
  cl_label_border<<<gc, 256, 0, s>>>(c->peaks, PK, ep, c->core, c->label);
  cl_zero_keys<<<gc, 256, 0, s>>>(PK, c->repkey);
  cl_repkey<<<gc, 256, 0, s>>>(c->peaks, PK, c->label, c->repkey, c->bm_r);
  e = scan_words(c->bm_r, c->rwords, c->pf_r, c->bsum, s);
  if (e != cudaSuccess) return cuda_rc(e);
  cl_gather_reps<<<gc, 256, 0, s>>>(c->peaks, PK, c->repkey, c->bm_r, c->pf_r,
                                    c->reps, c->rep_idx);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_rc(e);
  c->last = s;
  c->ran = true;
  return DDSP_OK;
}

// Counts of the last run after it finished: peaks, reps, error word.
static int cluster_counts(ddsp_cluster *c, uint32_t *n_peaks,
                          uint32_t *n_reps) {
  if (!c->ran) return DDSP_E_STATE;
  cudaError_t e = cudaStreamSynchronize(c->last);
  ClState st{};
  if (e == cudaSuccess) e = cudaMemcpy(&st, c->st, sizeof st, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess)
    e = cudaMemcpy(n_peaks, c->pf_p + c->nwords, 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess)
    e = cudaMemcpy(n_reps, c->pf_r + c->rwords, 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_rc(e);
  if (st.err & (kErrRecord | kErrRepeat)) return DDSP_E_INVALID_ARG;
  if (st.err & kErrLimit) return DDSP_E_TIMEOUT;
  return DDSP_OK;
}

extern "C" int ddsp_cluster_fetch_peaks(ddsp_cluster *c, ddsp_cand *host_peaks,
                                        int32_t *host_labels, size_t cap,
                                        size_t *n_peaks) {
  if (!c || !n_peaks || (cap > 0 && !host_peaks)) return DDSP_E_INVALID_ARG;
  DeviceGuard g(c->device);
  uint32_t np = 0, nr = 0;
  int rc = cluster_counts(c, &np, &nr);
  if (rc != DDSP_OK) return rc;
  *n_peaks = np;
  const size_t m = std::min<size_t>(np, cap);
  cudaError_t e = cudaSuccess;
  if (m > 0) {
    e = cudaMemcpy(host_peaks, c->peaks, m * sizeof(ddsp_cand),
                   cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && host_labels)
      e = cudaMemcpy(host_labels, c->label, m * 4, cudaMemcpyDeviceToHost);
  }
  if (e != cudaSuccess) return cuda_rc(e);
  return np > cap ? DDSP_E_TRUNCATED : DDSP_OK;
}

extern "C" int ddsp_cluster_fetch_reps(ddsp_cluster *c, ddsp_cand *host_reps,
                                       uint32_t *host_idx, size_t cap,
                                       size_t *n_reps) {
  if (!c || !n_reps || (cap > 0 && !host_reps)) return DDSP_E_INVALID_ARG;
  DeviceGuard g(c->device);
  uint32_t np = 0, nr = 0;
  int rc = cluster_counts(c, &np, &nr);
  if (rc != DDSP_OK) return rc;
  *n_reps = nr;
  const size_t m = std::min<size_t>(nr, cap);
  cudaError_t e = cudaSuccess;
  if (m > 0) {
    e = cudaMemcpy(host_reps, c->reps, m * sizeof(ddsp_cand),
                   cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && host_idx)
      e = cudaMemcpy(host_idx, c->rep_idx, m * 4, cudaMemcpyDeviceToHost);
  }
  if (e != cudaSuccess) return cuda_rc(e);
  return nr > cap ? DDSP_E_TRUNCATED : DDSP_OK;
}

extern "C" int ddsp_plan_candidates_device(ddsp_plan *h,
                                           const ddsp_cand **d_cands,
                                           const uint32_t **d_count,
                                           size_t *capacity) {
  if (!h || !d_cands || !d_count || !capacity) return DDSP_E_INVALID_ARG;
  *d_cands = h->p.d_cands;
  *d_count = h->p.d_count;
  *capacity = h->p.cand_capacity;
  return DDSP_OK;
}
