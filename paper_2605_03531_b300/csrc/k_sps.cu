// k_sps.cu -- boxcar single-pulse search (Sec.2.1) with the robust median /
// MAD noise estimate of Sec.3.3, fused into one kernel: one block per
// (DM trial k, normalisation window j).
//
//   1. load the window x[lo, hi) plus (w_max - 1) samples of look-ahead into
//      shared memory (the series is read from HBM once);
//   2. exact median and MAD of the window on integer keys: in one pass of
//      4096 single-value bins around an estimate from 32 sorted samples
//      when the window's middle half is narrow (median_fast, mad_fast_warp), else by
//      histogram selection: a 2048-bin shared histogram over the current
//      key range narrows it by 2^11 per pass until the bin holding the
//      wanted order statistic is one key wide (or the two middle order
//      statistics fall in different bins: then max of the lower bin and min
//      of the upper bin); m2 = 2*median, mad4 = 4*MAD are exact integers;
//   3. an exclusive prefix sum Q in uint32 (modular, so every difference
//      Q[t+w] - Q[t] is exact) of y = 2x - m2 when the window keeps every
//      S/N numerator 2 B_y - w*odd below 2^30 in magnitude (a difference is
//      then the numerator itself), else of y = x - floor(median) (a
//      difference is B_y = B_w(t) - w*floor(median)), computed with
//      warp-shuffle scans, recording per chunk of 8 start times the
//      extremes of Q and the largest y;
//   4. per chunk a bound of every width's boxcar sums from those extremes
//      against the integer screen thresholds (derived from the S/N
//      threshold with a small safety margin); only chunks that could pass
//      go start by start through the exact path: the FP32 S/N of every
//      width, the best one (first maximum), and candidate emission through
//      a per-warp stage in shared memory, one atomicAdd on the global count
//      per stage-full (ballot + popc place the records).
// Memory traffic is 4 bytes per series sample read once (plus the look-ahead)
// and 16 bytes per candidate: the kernel is bounded by HBM bandwidth.
#include <math.h>

#include "dev_util.cuh"
#include "internal.h"

namespace ddsp {
namespace {

constexpr int kSpsThreads = 256;  // four blocks per SM
constexpr int kWarps = kSpsThreads / 32;
constexpr int kBins = 2048;      // bins per pass of the generic selection
constexpr int kSelPer = kBins / kSpsThreads;
constexpr int kFastBins = 4096;  // single-value bins of the one-pass path
constexpr int kMaxWidths = 11;  // 1 .. 1024
constexpr int64_t kMaxWindowSamples = 49152;
constexpr float kMadToSigma = 1.482602218505602f;

struct SpsShared {
  uint32_t hist[kFastBins + 32];  // + a sink per lane for keys outside the bins
  uint32_t wred[kWarps][2];
  uint32_t hred[kWarps][2];
  uint32_t wsx[kWarps];    // each warp's sum of x over its scan groups
  uint32_t nbw[kWarps];    // each warp's count of keys below the bins
  int64_t bc[6];      // broadcast slots
  float inv[kMaxWidths];
  int32_t thr_by[kMaxWidths];
  int32_t wid[kMaxWidths];
  uint32_t wsum[kWarps];
};

// The window buffer follows the struct, 16-byte aligned (vector accesses).
constexpr size_t kBufOff = (sizeof(SpsShared) + 15) & ~(size_t)15;

// Inclusive warp scan (Hillis-Steele): the shuffle's own predicate says
// whether lane - o exists, so each step is one shuffle and one predicated
// add.
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane) {
  (void)lane;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    asm("{\n\t.reg .u32 t;\n\t.reg .pred p;\n\t"
        "shfl.sync.up.b32 t|p, %0, %1, 0, 0xffffffff;\n\t"
        "@p add.u32 %0, %0, t;\n\t}"
        : "+r"(v)
        : "r"(o));
  }
  return v;
}

// float(d) for |d| < 2^22, exact: the integer added to the bit pattern of
// 1.5 * 2^23 (whose unit in the last place is 1) and the constant taken
// away again, two full-rate operations instead of a conversion.
__device__ __forceinline__ float small_int_to_float(int32_t d) {
  return __int_as_float(0x4B400000 + d) - 12582912.0f;
}

// float(2*by - c), rounded to nearest, for any int32 by and 0 <= c < 2^16,
// without a 64-bit integer conversion: 2*by - c = hi*2^17 + lo with
// hi = by >> 16 and lo = 2*(by & 0xffff) - c; both parts (|.| < 2^22) are
// converted exactly by the 1.5*2^23 magic-number trick and one fused
// multiply-add rounds their exact sum once.
__device__ __forceinline__ float twice_minus(int32_t by, int32_t c) {
  const int32_t hi = by >> 16;
  const int32_t lo = 2 * (by & 0xffff) - c;
  const float hf = small_int_to_float(hi);
  const float lf = small_int_to_float(lo);
  return __fmaf_rn(hf, 131072.0f, lf);
}

// Sum of wsum[0 .. warp-1] (kWarps <= 32 per-warp totals), by one warp scan.
__device__ __forceinline__ uint32_t warp_excl_offset(const uint32_t *wsum,
                                                     int warp, int lane) {
  const uint32_t v = lane < kWarps ? wsum[lane] : 0u;
  const uint32_t inc = warp_incl_scan(v, lane);
  const uint32_t below = __shfl_sync(0xffffffffu, inc, warp > 0 ? warp - 1 : 0);
  return warp > 0 ? below : 0u;
}

// Exact order statistics of rank r1 and r2 = r1 or r1 + 1 (0-based) of n
// uint32 keys produced by key(i), all <= kmax.  Returns them in k1, k2.
template <typename KeyFn>
__device__ void select2(KeyFn key, int n, int r1, int r2, uint32_t kmax,
                        SpsShared &sh, uint32_t &k1, uint32_t &k2) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t lo = 0;
  uint64_t span = (uint64_t)kmax + 1;
  int below = 0;
  while (true) {
    int s = 0;
    while (((span - 1) >> s) >= (uint64_t)kBins) ++s;
    const int nb = (int)((span - 1) >> s) + 1;
    for (int b = tid; b < nb; b += kSpsThreads) sh.hist[b] = 0;
    __syncthreads();
    const uint32_t smax = (uint32_t)(span - 1);   // span <= 2^32
    for (int i = tid; i < n; i += kSpsThreads) {
      const uint32_t k = key(i);
      const uint32_t d = k - lo;
      if (k >= lo && d <= smax) atomicAdd(&sh.hist[d >> s], 1u);
    }
    __syncthreads();
    // exclusive scan of the histogram: each thread owns kSelPer
    // consecutive bins
    uint32_t c[kSelPer], tsum = 0;
#pragma unroll
    for (int q = 0; q < kSelPer; ++q) {
      int b = kSelPer * tid + q;
      c[q] = (b < nb) ? sh.hist[b] : 0;
      tsum += c[q];
    }
    uint32_t incl = warp_incl_scan(tsum, lane);
    if (lane == 31) sh.wsum[warp] = incl;
    __syncthreads();
    const uint32_t wpre = warp_excl_offset(sh.wsum, warp, lane);
    // keys of this window below bin kSelPer * tid
    uint32_t run = wpre + incl - tsum;
    const uint32_t q1 = (uint32_t)(r1 - below), q2 = (uint32_t)(r2 - below);
#pragma unroll
    for (int q = 0; q < kSelPer; ++q) {
      int b = kSelPer * tid + q;
      if (b < nb && c[q] > 0) {
        if (q1 >= run && q1 < run + c[q]) {
          sh.bc[0] = b;
          sh.bc[2] = run;
        }
        if (q2 >= run && q2 < run + c[q]) {
          sh.bc[1] = b;
          sh.bc[3] = run;
        }
      }
      run += c[q];
    }
    __syncthreads();
    const int b1 = (int)sh.bc[0], b2 = (int)sh.bc[1];
    const int run1 = (int)sh.bc[2];
    __syncthreads();
    if (s == 0) {
      k1 = lo + (uint32_t)b1;
      k2 = lo + (uint32_t)b2;
      return;
    }
    if (b1 == b2) {
      below += run1;
      lo += (uint32_t)b1 << s;
      uint64_t rest = span - ((uint64_t)b1 << s);
      span = min((uint64_t)1 << s, rest);
      continue;
    }
    // r2 = r1 + 1 sits in a later bin: k1 = max of bin b1, k2 = min of bin b2
    uint32_t mx = 0, mn = 0xffffffffu;
    const uint32_t smax2 = (uint32_t)(span - 1);
    for (int i = tid; i < n; i += kSpsThreads) {
      const uint32_t k = key(i);
      const uint32_t d = k - lo;
      if (k >= lo && d <= smax2) {
        int b = (int)(d >> s);
        if (b == b1) mx = max(mx, k);
        if (b == b2) mn = min(mn, k);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    }
    if (lane == 0) {
      sh.wred[warp][0] = mx;
      sh.wred[warp][1] = mn;
    }
    __syncthreads();
    if (tid == 0) {
      uint32_t a = 0, b = 0xffffffffu;
      for (int w = 0; w < kWarps; ++w) {
        a = max(a, sh.wred[w][0]);
        b = min(b, sh.wred[w][1]);
      }
      sh.bc[0] = a;
      sh.bc[1] = b;
    }
    __syncthreads();
    k1 = (uint32_t)sh.bc[0];
    k2 = (uint32_t)sh.bc[1];
    __syncthreads();
    return;
  }
}

// The estimate the one-pass bins start from: 32 evenly spaced samples of the
// window [0, n), read straight from global memory by one warp (while the
// other warps load the window) and sorted in that warp; bc[0] = their median
// (a sample value), bc[1] = their interquartile range, bc[2 .. 5] = -1.
__device__ __forceinline__ void median_estimate(const int32_t *__restrict__ x,
                                                int64_t lo, int64_t n_series,
                                                int n, SpsShared &sh) {
  const int lane = threadIdx.x & 31;
  const int i = (lane * n) >> 5;   // n < 2^26
  int32_t v = 0;
  if (DDSP_BC(lo + i < n_series, kBcSpsLoad, lo + i)) v = __ldg(x + i);
#pragma unroll
  for (int kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
    for (int jj = kk >> 1; jj > 0; jj >>= 1) {
      const int32_t o = __shfl_xor_sync(0xffffffffu, v, jj);
      const bool up = (lane & kk) == 0, low = (lane & jj) == 0;
      v = (low == up) ? min(v, o) : max(v, o);
    }
  }
  const int32_t med = __shfl_sync(0xffffffffu, v, 16);
  const int32_t q1 = __shfl_sync(0xffffffffu, v, 8);
  const int32_t q3 = __shfl_sync(0xffffffffu, v, 24);
  if (lane == 0) {
    sh.bc[0] = med;
    sh.bc[1] = (int64_t)q3 - (int64_t)q1;
#pragma unroll
    for (int q = 2; q < 6; ++q) sh.bc[q] = -1;
  }
}

// Exact median and MAD from one histogram pass, for windows whose middle
// half is narrow: keys k = x - min, ranks r1 <= r2 = r1 or r1 + 1.
//  * the load (step 1) counted every window sample in single-value bins of
//    keys [A, A + 4096) around an estimate (median_estimate: 32 evenly spaced
//    samples give the median and the quartiles; wide windows, estimated
//    IQR > 2800, go to select2) and, per warp, the samples below A (nbw);
//    A may be negative (bins below the window's minimum stay empty);
//  * their prefix sums P give the two middle order statistics k1, k2
//    directly;
//  * with m = k1 + k2 (= M2 - 2*min), #{|2k - m| <= v} is the number of
//    keys in [ceil((m - v)/2), floor((m + v)/2)], a difference of two prefix
//    sums while that range lies inside the bins (or starts below them when
//    no key is below the bins); the MAD order statistics are the smallest v
//    reaching ranks r1 + 1 and r2 + 1.
// A rank outside the bins sends that part to select2 (the median at once,
// the MAD after the scan); the results equal select2's.
// median_fast: the median part (block-wide), true with k1, k2 and the
// count below the bins when both middle ranks fall inside them; the prefix
// P stays in the bins for mad_fast_warp.
__device__ bool median_fast(int64_t A, int r1, int r2, SpsShared &sh,
                            uint32_t &k1, uint32_t &k2, uint32_t &below_out) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t below = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) below += sh.nbw[w];
  // ---- inclusive prefix P[b] = below + #{keys in [A, A + b]}, in place.
  // Warp w owns bins [kWarpBins w, kWarpBins (w + 1)) and lane l the four
  // bins 4l .. 4l + 3 of each 128-bin segment of them, so every 16-byte
  // shared access of a warp touches 512 consecutive bytes (no bank
  // conflicts): the warps' totals first, then the prefix with every warp's
  // offset known, and the median ranks found on the way.
  constexpr int kWarpBins = kFastBins / kWarps;
  constexpr int kSegs = kWarpBins / 128;
  uint32_t *wbins = sh.hist + kWarpBins * warp + 4 * lane;
  uint4 cnt[kSegs];
  uint32_t wtot = 0;
#pragma unroll
  for (int sg = 0; sg < kSegs; ++sg) {
    cnt[sg] = *reinterpret_cast<const uint4 *>(wbins + 128 * sg);
    wtot += cnt[sg].x + cnt[sg].y + cnt[sg].z + cnt[sg].w;
  }
  wtot = __reduce_add_sync(0xffffffffu, wtot);
  if (lane == 0) sh.wsum[warp] = wtot;
  __syncthreads();
  uint32_t run = below + warp_excl_offset(sh.wsum, warp, lane);
  const uint32_t R1 = (uint32_t)r1 + 1u, R2 = (uint32_t)r2 + 1u;
  // ---- median: the smallest b with P[b] >= r + 1
  auto hit = [&](uint32_t prev, uint32_t cur, int b) {
    if (prev < R1 && R1 <= cur) sh.bc[2] = b;
    if (prev < R2 && R2 <= cur) sh.bc[3] = b;
  };
#pragma unroll
  for (int sg = 0; sg < kSegs; ++sg) {
    const uint4 c = cnt[sg];
    const uint32_t t = c.x + c.y + c.z + c.w;
    const uint32_t inc = warp_incl_scan(t, lane);
    const uint32_t pre = run + inc - t;
    const uint32_t p0 = pre + c.x, p1 = p0 + c.y, p2 = p1 + c.z, p3 = p2 + c.w;
    // a rank reached inside this lane's four bins (R1 <= R2): rare, so the
    // bins are told apart only then
    if (pre < R2 && R1 <= p3) {
      const int b0 = kWarpBins * warp + 128 * sg + 4 * lane;
      hit(pre, p0, b0);
      hit(p0, p1, b0 + 1);
      hit(p1, p2, b0 + 2);
      hit(p2, p3, b0 + 3);
    }
    *reinterpret_cast<uint4 *>(wbins + 128 * sg) = make_uint4(p0, p1, p2, p3);
    run += __shfl_sync(0xffffffffu, inc, 31);
  }
  __syncthreads();
  // (nothing writes bc[2], bc[3] again in this window, and select2, if it
  // follows, starts with a barrier: no barrier after these reads)
  const int64_t b1 = sh.bc[2], b2 = sh.bc[3];
  if (b1 < 0 || b2 < 0) return false;  // block-uniform
  k1 = (uint32_t)(A + b1);
  k2 = (uint32_t)(A + b2);
  below_out = below;
  return true;
}

// mad_fast_warp: the MAD part, run by warps 0 and 1 only (one rank each,
// no block barrier, so the other warps go on meanwhile): bc[4 + warp] =
// the rank's order statistic of |2k - m|, or -1 when it leaves the bins.
__device__ void mad_fast_warp(int64_t A, uint32_t below, uint32_t k1,
                              uint32_t k2, int r1, int r2, SpsShared &sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // ---- MAD: C(v) = #{|2k - m| <= v}, -1 when its key range leaves the bins
  const int64_t m = (int64_t)k1 + (int64_t)k2;
  const int64_t lo_ok = A, hi_ok = A + kFastBins - 1;
  auto count_within = [&](int64_t v) -> int64_t {
    const int64_t lo = (m - v + 1) >> 1, hi = (m + v) >> 1;
    if (hi > hi_ok || (lo < lo_ok && lo_ok > 0)) return -1;
    const int64_t ph = sh.hist[hi - lo_ok];
    // no key lies below min (key 0), so none below lo <= A <= 0 either
    const int64_t pl = lo <= lo_ok ? (lo == lo_ok ? (int64_t)below : 0)
                                   : (int64_t)sh.hist[lo - lo_ok - 1];
    return ph - pl;
  };
  // C is non-decreasing in v and valid on a prefix of [0, 2 * kFastBins),
  // so the smallest v with C(v) >= R is found by one warp per rank in
  // three 32-way steps of widths 256, 8 and 1, each lane testing the last
  // v of its part.
  static_assert(2 * kFastBins == 32 * 256, "MAD search covers [0, 8192)");
  {
    const int which = warp;
    const int64_t R = (int64_t)(which ? r2 : r1) + 1;
    int64_t base = 0;
    bool found = true;
#pragma unroll
    for (int st = 0; st < 3; ++st) {
      const int64_t w = st == 0 ? 256 : (st == 1 ? 8 : 1);
      const int nl = st == 2 ? 8 : 32;
      const int64_t cv = lane < nl ? count_within(base + lane * w + w - 1) : -1;
      const unsigned hit = __ballot_sync(0xffffffffu, cv >= R);
      if (hit == 0u) {   // warp-uniform: only possible in the first step
        found = false;
        break;
      }
      base += (int64_t)(__ffs(hit) - 1) * w;
    }
    if (lane == 0) sh.bc[4 + which] = found ? base : -1;
  }
}

// Chunk bounds of the screen.  Start times are taken in chunks of kChunk;
// per chunk c the scan records the smallest and largest prefix value
// Q[8c .. 8c+7] and the largest y[8c .. 8c+7].  For every start i of chunk
// c and width w, B_w(i) = Q[i + w] - Q[i] is at most the largest Q over the
// chunks holding [8c + w, 8c + w + 8) minus the smallest Q of chunk c, and
// also at most w times the largest y over [8c, 8c + 7 + w); a chunk none of
// whose widths can reach its integer threshold is skipped without looking
// at its starts.  On noise that rejects all but a few chunks in a thousand,
// so the screen costs a few operations per sample instead of one load, add
// and compare per sample and width.
constexpr int kChunk = 8;
// prefix positions per scan group: 32 lanes x one chunk each
constexpr int kGroup = 32 * kChunk;
// windows up to this many buffered samples keep the chunk statistics in
// shared memory (longer ones take every start through the exact screen)
constexpr int64_t kStatsMaxCap = 32768;
// Windows longer than the on-chip limit (long mode): exact statistics by a
// separate pass over global memory, then the search in segments of kSeg
// start times (each with its look-ahead), all of a window sharing them.
constexpr int64_t kSeg = 8192;

__host__ __device__ __forceinline__ int64_t sps_buf_cap(int64_t maxlen,
                                                        int wmax) {
  // x[0 .. elen) then, in place, Q[0 .. elen]; rounded to whole
  // 256-position scan groups
  return ((maxlen + wmax + 1 + 255) / 256) * 256;
}
__host__ __device__ __forceinline__ int64_t sps_chunk_cap(int64_t cap) {
  return cap / kChunk + 2;
}

// One start time through the exact path: the boxcar differences of every
// width from the prefix values, the FP32 S/N and the best width (first
// maximum).  Q2: the prefix is of y2 = 2x - M2, so a difference is the S/N
// numerator 2 B_y - w*odd itself, below 2^22 in magnitude, and two
// full-rate operations convert it exactly; else the prefix is of
// y = x - floor(median), a difference is B_y and twice_minus rounds
// 2 B_y - w*odd (no conversion instruction either: on this GPU it issues
// at a fraction of the integer and FP32 rate).  Returns the best
// width index (-1: none) with its S/N and its difference.
// NW > 0: the widths are 1, 2, 4, ..., 2^(NW-1), so the boxcar ends are
// compile-time offsets and a start whose widest boxcar ends inside the
// series needs no per-width check; every width's S/N is taken (the same
// best comes out as from the widths that pass the integer screen: a width
// that fails it has S/N below the threshold, so it can be the best only
// when no width reaches the threshold and there is no candidate either
// way).  NW = 0: any ascending width list, each width screened first
// (every width in the dense mode).
template <bool DENSE, int NW, bool Q2, bool N32 = false>
__device__ __forceinline__ int exact_start(
    const uint32_t *__restrict__ Q, int qcap, int i, int nv, int nw,
    const int32_t (&wv)[kMaxWidths], const int32_t (&tbv)[kMaxWidths],
    const float (&iv)[kMaxWidths], int odd, float &bs, int32_t &bd) {
  const uint32_t qi = Q[i];
  int bw = -1;
  bs = 0.0f;
  bd = 0;
  if constexpr (NW > 0) {
    constexpr int kWidest = 1 << (NW - 1);
    const bool inner = i + kWidest <= nv &&
                       DDSP_BC(i + kWidest < qcap, kBcSpsQ, i + kWidest);
    // every width's S/N (-inf for a boxcar past the series end), then the
    // first maximum by a pairwise tree: the right group (higher widths) wins
    // only when strictly larger, so ties keep the lowest width, as a scan
    // in width order would, with log2(NW) dependent steps instead of NW
    float sn[NW];
    int32_t dd[NW];
    int id[NW];
#pragma unroll
    for (int wi = 0; wi < NW; ++wi) {
      const bool v = inner || (i + (1 << wi) <= nv &&
                               DDSP_BC(i + (1 << wi) < qcap, kBcSpsQ, i));
      id[wi] = wi;
      dd[wi] = 0;
      sn[wi] = -INFINITY;
      if (v) {
        dd[wi] = (int32_t)(Q[i + (1 << wi)] - qi);
        // N32 (y prefix): widths up to 32 keep 2 B_y - w*odd below 2^22,
        // so it converts exactly by two operations as well
        sn[wi] = (Q2 ? small_int_to_float(dd[wi])
                  : (N32 && (1 << wi) <= 32)
                      ? small_int_to_float(2 * dd[wi] - (odd << wi))
                      : twice_minus(dd[wi], odd << wi)) *
                 iv[wi];
      }
    }
#pragma unroll
    for (int st = 1; st < NW; st <<= 1) {
#pragma unroll
      for (int a = 0; a + st < NW; a += 2 * st) {
        const bool right = sn[a + st] > sn[a];
        sn[a] = right ? sn[a + st] : sn[a];
        id[a] = right ? id[a + st] : id[a];
        dd[a] = right ? dd[a + st] : dd[a];
      }
    }
    if (sn[0] != -INFINITY) {   // (width 1 always fits: never taken here)
      bw = id[0];
      bs = sn[0];
      bd = dd[0];
    }
  } else {
#pragma unroll
    for (int wi = 0; wi < kMaxWidths; ++wi) {
      if (wi < nw && i + wv[wi] <= nv &&
          DDSP_BC(i + wv[wi] < qcap, kBcSpsQ, i + wv[wi])) {
        const int32_t d = (int32_t)(Q[i + wv[wi]] - qi);
        if (DENSE || d >= tbv[wi]) {
          const float sn =
              (Q2 ? small_int_to_float(d) : twice_minus(d, wv[wi] * odd)) *
              iv[wi];
          if (bw < 0 || sn > bs) {
            bw = wi;
            bs = sn;
            bd = d;
          }
        }
      }
    }
  }
  return bw;
}

// Candidate emission.  Each warp appends its candidates to its own stage
// in shared memory, one word a record (start << 4 | width index; ballot +
// popc give the positions), and, when the next run might not fit and at
// the end of the window, moves the stage to the output with one atomicAdd
// on the global count and coalesced 16-byte stores, each record's S/N
// recomputed from the prefix values with the operations that produced it
// (the same bits); records beyond the capacity are dropped, the count
// stays exact.  Without room for a stage of 32 records (scap == 0) every
// run reserves its own slots.
struct Emitter {
  uint32_t *stage;   // this warp's stage: scap words
  int scap;          // records it holds (0: no stage)
  int n;             // records staged (warp-uniform)
};

// rec(word) -> ddsp_cand rebuilds a staged record.
template <typename RecFn>
__device__ __forceinline__ void emit_flush(Emitter &e, RecFn rec,
                                           ddsp_cand *__restrict__ cands,
                                           uint32_t *__restrict__ count,
                                           uint32_t cap) {
  const int lane = threadIdx.x & 31;
  if (e.n == 0) return;                         // warp-uniform
  __syncwarp();
  uint32_t base = 0;
  if (lane == 0) base = atomicAdd(count, (uint32_t)e.n);
  base = __shfl_sync(0xffffffffu, base, 0);
  for (int r = lane; r < e.n; r += 32)
    if (base + (uint32_t)r < cap) cands[base + (uint32_t)r] = rec(e.stage[r]);
  __syncwarp();
  e.n = 0;
}

// The candidates of one run of 32 starts (all lanes of the warp call it).
template <typename RecFn>
__device__ __forceinline__ void emit(Emitter &e, bool cand, int k, int64_t lo,
                                     int i, int bw, float bs, RecFn rec,
                                     ddsp_cand *__restrict__ cands,
                                     uint32_t *__restrict__ count,
                                     uint32_t cap) {
  const int lane = threadIdx.x & 31;
  const unsigned ball = __ballot_sync(0xffffffffu, cand);
  if (ball == 0u) return;                       // warp-uniform
  const int nb = __popc(ball);
  const uint32_t below = __popc(ball & ((1u << lane) - 1u));
  if (e.scap == 0) {
    const int leader = __ffs(ball) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(count, (uint32_t)nb);
    base = __shfl_sync(0xffffffffu, base, leader);
    if (cand && base + below < cap) {
      ddsp_cand c;
      c.dm_idx = (uint32_t)k;
      c.t = (uint32_t)(lo + i);
      c.w_idx = (uint32_t)bw;
      c.snr = bs;
      cands[base + below] = c;
    }
    return;
  }
  if (e.n + nb > e.scap) emit_flush(e, rec, cands, count, cap);
  if (cand) e.stage[e.n + (int)below] = ((uint32_t)i << 4) | (uint32_t)bw;
  e.n += nb;
}

// What the sweep of one window needs (step 4).
struct SweepArgs {
  const uint32_t *Q;
  int qcap, len, nv, nw, odd;
  int32_t mfloor;
  int64_t m2;
  float thr;
  int64_t lo, n, nrep;
  int k, wmax;
  bool bounds;
  const int32_t *cmin, *cmax, *ymax;
  const int32_t *wid;       // the widths (shared memory)
  const float *inv;         // their S/N scales (shared memory)
  uint32_t *stage;          // the warps' stages (shared memory)
  int scap;                 // records per warp stage (0: none)
  ddsp_cand *cands;
  uint32_t *count;
  uint32_t cap;
  int32_t *best_w;
  float *best_snr;
  int32_t *best_sum;
};

// Step 4: boxcars, S/N, candidates of one window (NW and Q2 as in
// exact_start).
template <bool DENSE, int NW, bool Q2, bool N32 = false>
__device__ __forceinline__ void sweep(const SweepArgs &g,
                                      const int32_t (&wv)[kMaxWidths],
                                      const int32_t (&tbv)[kMaxWidths],
                                      const float (&iv)[kMaxWidths],
                                      int64_t bufcap) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (DENSE) {
    for (int i = tid; i < g.len; i += kSpsThreads) {
      float bs;
      int32_t bd;
      const int bw = exact_start<true, NW, Q2, N32>(g.Q, g.qcap, i, g.nv, g.nw, wv,
                                               tbv, iv, g.odd, bs, bd);
      // the boxcar sum of x: (num + w*M2)/2 (Q2) or B_y + w*floor(median),
      // modulo 2^32
      int32_t bsum = 0;
      if (bw >= 0) {
        const int w = NW > 0 ? (1 << bw) : g.wid[bw];
        bsum = Q2 ? (int32_t)(((int64_t)bd + (int64_t)w * g.m2) >> 1)
                  : (int32_t)((uint32_t)bd + (uint32_t)w * (uint32_t)g.mfloor);
      }
      const int64_t o = (int64_t)g.k * g.n + g.lo + i;
      if (DDSP_BC(g.lo + i < g.n, kBcSpsDense, g.lo + i)) {
        g.best_w[o] = bw;
        g.best_snr[o] = bs;
        g.best_sum[o] = bsum;
      }
    }
    return;
  }
  Emitter em{g.stage + g.scap * warp, g.scap, 0};
  // a staged record back to its output form: the S/N of width bw at start
  // i, computed as exact_start computes it
  auto rec = [&](uint32_t word) {
    const int i = (int)(word >> 4), bw = (int)(word & 15u);
    const int w = NW > 0 ? (1 << bw) : g.wid[bw];
    const int32_t d = (int32_t)(g.Q[i + w] - g.Q[i]);
    ddsp_cand c;
    c.dm_idx = (uint32_t)g.k;
    c.t = (uint32_t)(g.lo + i);
    c.w_idx = (uint32_t)bw;
    c.snr = (Q2 ? small_int_to_float(d)
             : (N32 && w <= 32) ? small_int_to_float(2 * d - w * g.odd)
                                : twice_minus(d, w * g.odd)) *
            g.inv[bw];
    return c;
  };
  // A warp takes 32 consecutive chunks (256 start times) at a time: lane l
  // bounds chunk l; the chunks that could pass then go through the exact
  // path 32 consecutive starts at a time, one per lane (consecutive
  // shared-memory words: no bank conflicts), skipping the 32-start runs
  // whose four chunks all failed their bounds.
  const int nch = (g.len + kChunk - 1) / kChunk;
  for (int cb = warp * 32; cb < nch; cb += kSpsThreads) {
    const int c = cb + lane;
    bool need = false;
    if (c < nch) {
      const int i0 = c * kChunk;
      need = true;
      if (g.bounds && i0 + kChunk + g.wmax <= g.nv &&
          DDSP_BC((c + g.wmax / kChunk + 1) < sps_chunk_cap(bufcap),
                  kBcSpsBound, c)) {
        const int32_t lmin = g.cmin[c];
        const int32_t ym1 = g.ymax[c];
        const int32_t ym2 = max(ym1, g.ymax[c + 1]);
        bool pass = false;
#pragma unroll
        for (int wi = 0; wi < kMaxWidths; ++wi) {
          if (NW > 0 ? wi < NW : wi < g.nw) {
            const int w = NW > 0 ? (1 << wi) : wv[wi];
            const int c2 = c + w / kChunk;
            int32_t top = g.cmax[c2];
            if (w % kChunk) top = max(top, g.cmax[c2 + 1]);
            // |Q| < 2^30 here, so the difference is exact in int32
            int32_t ub = top - lmin;
            if (w < kChunk) {
              // w * max y fits: |y| (elen + 1) < 2^30 and w < 8 <= elen
              const int32_t yb = w * (w == 1 ? ym1 : ym2);
              ub = min(ub, yb);
            }
            pass |= ub >= tbv[wi];
          }
        }
        need = pass;
      }
    }
    const unsigned pm = __ballot_sync(0xffffffffu, need);
    if (pm == 0u) continue;                      // warp-uniform
#pragma unroll 1
    for (int sb = 0; sb < kChunk; ++sb) {        // 8 runs of 32 starts
      // starts [8 cb + 32 sb, + 32): chunks cb + 4 sb .. cb + 4 sb + 3
      const unsigned sub = (pm >> (4 * sb)) & 0xFu;
      if (sub == 0u) continue;                   // warp-uniform
      const int i = kChunk * cb + 32 * sb + lane;
      const bool mine = ((sub >> (lane >> 3)) & 1u) && i < g.len;
      float bs = 0.0f;
      int32_t bd;
      int bw = -1;
      if (mine)
        bw = exact_start<false, NW, Q2, N32>(g.Q, g.qcap, i, g.nv, g.nw, wv, tbv,
                                        iv, g.odd, bs, bd);
      const bool cand = bw >= 0 && bs >= g.thr && g.lo + i < g.nrep;
      emit(em, cand, g.k, g.lo, i, bw, bs, rec, g.cands, g.count, g.cap);
    }
  }
  emit_flush(em, rec, g.cands, g.count, g.cap);
}

// The search of one (DM trial k, window j): the body of the per-plan kernel
// and of the multi-beam kernel (k_batch.cu).  Shared memory: SpsShared, then
// buf[bufcap] (x, then Q in place), then, for bufcap <= kStatsMaxCap, the
// chunk statistics cmin / cmax / ymax [sps_chunk_cap(bufcap)] each.
template <bool DENSE>
__device__ __forceinline__ void sps_window(
    const int32_t *__restrict__ series, int64_t n, int64_t L, int64_t nwin,
    const int32_t *__restrict__ widths, int nw, float thr,
    int64_t *__restrict__ m2_out, int64_t *__restrict__ mad4_out,
    ddsp_cand *__restrict__ cands, uint32_t *__restrict__ count, uint32_t cap,
    int32_t *__restrict__ best_w, float *__restrict__ best_snr,
    int32_t *__restrict__ best_sum, int32_t *__restrict__ err,
    const int64_t j, const int k, const int64_t nrep, const int64_t bufcap,
    const int64_t seg = -1) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SpsShared &sh = *reinterpret_cast<SpsShared *>(smem_raw);
  int32_t *buf = reinterpret_cast<int32_t *>(smem_raw + kBufOff);
  // chunk statistics: in the histogram's space when they fit (the
  // histogram is done before the scan writes them), else after the buffer
  const int64_t ccap = sps_chunk_cap(bufcap);
  const bool stats_in_hist = 3 * ccap <= kFastBins;
  const bool have_stats = stats_in_hist || bufcap <= kStatsMaxCap;
  int32_t *cmin = stats_in_hist ? reinterpret_cast<int32_t *>(sh.hist)
                                : buf + bufcap;
  int32_t *cmax = cmin + ccap;
  int32_t *ymax = cmax + ccap;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // seg < 0: the whole window j, its statistics computed here; seg >= 0
  // (long windows): start times [lo, hi) = segment seg of kSeg samples of
  // window j, whose statistics sps_long_stats_kernel already wrote
  const bool given = seg >= 0;
  const int64_t wlo = (L <= 0) ? 0 : j * L;
  const int64_t whi = (L <= 0 || j == nwin - 1) ? n : (j + 1) * L;
  const int64_t lo = given ? wlo + seg * kSeg : wlo;
  const int64_t hi = given ? min(lo + kSeg, whi) : whi;
  const int wmax = widths[nw - 1];
  const int64_t ext = min(hi + wmax - 1, n);
  const int len = (int)(hi - lo), elen = (int)(ext - lo);
  const int32_t *x = series + (int64_t)k * n + lo;

  // ---- 1. load x[0 .. elen) to buf, min and max over the window [0, len)
  // and over the look-ahead [len, elen), each warp's sum of x over its run
  // of the scan's 128-position groups (so step 3 needs one pass), and the
  // median's histogram of the window (step 2's one-pass bins, filled as the
  // samples arrive).  A lane takes 4 consecutive samples of a group: 16-byte
  // loads when the window starts on a 16-byte boundary (n and L multiples
  // of 4).
  int32_t mn32 = INT32_MAX, mx32 = INT32_MIN;   // the window [0, len)
  int32_t hmn = INT32_MAX, hmx = INT32_MIN;     // look-ahead [len, elen)
  auto take = [&](int i, int32_t v) {
    if (i < len) {
      mn32 = min(mn32, v);
      mx32 = max(mx32, v);
    } else {
      hmn = min(hmn, v);
      hmx = max(hmx, v);
    }
  };
  const int ntot = elen + 1;                    // prefix positions 0 .. elen
  const int ngroups = (ntot + kGroup - 1) / kGroup;
  const int gpw = (ngroups + kWarps - 1) / kWarps;
  // warp w takes run kWarps - 1 - w of gpw groups: the runs at the end are
  // the short ones, so warps 0 and 1, which also estimate the median and
  // search the MAD, carry the least of the load and the scan
  const int run = kWarps - 1 - warp;
  const int g0 = run * gpw, g1 = min(ngroups, g0 + gpw);
  const bool vec = (reinterpret_cast<uintptr_t>(x) & 15) == 0;
  uint32_t sx = 0;                              // this lane's sum of x
  int h = 2 * g0;                               // 128-position halves
  // halves wholly inside the window proper go four at a time, four loads
  // in flight a lane; the first four leave before the estimate's barrier
  const int hin = vec ? min(2 * g1, len / 128) : h;
  auto batch_ok = [&](int hh) {
    return hh + 4 <= hin &&
           DDSP_BC((hh + 4) * 128 <= bufcap && lo + (hh + 4) * 128 <= n,
                   kBcSpsLoad, lo + hh * 128);
  };
  int4 v[4];
  bool have = batch_ok(h);
  if (have) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
      v[u] = __ldg(reinterpret_cast<const int4 *>(x + (h + u) * 128) + lane);
  }
  // the median estimate (warp 0 has the fewest load groups) and the
  // zeroed histogram, both visible after the barrier
  if (!given && warp == 0) median_estimate(x, lo, n, len, sh);
  for (int b = tid; b < (kFastBins + 32) / 4; b += kSpsThreads)
    reinterpret_cast<uint4 *>(sh.hist)[b] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  // Single-value bins [AB, AB + kFastBins) of x around the estimate and the
  // count of window samples below AB, for windows whose estimated
  // interquartile range is narrow (else step 2 goes to select2).  d = x - AB
  // mod 2^32 bins a sample and, by its top bit, counts it below the bins;
  // that holds while every x - AB lies in [-2^31, 2^31), which step 2
  // checks against the window's extremes before it trusts the counts.
  const bool binning = !given && sh.bc[1] <= 2800;   // block-uniform
  const int64_t AB64 = max((int64_t)(int32_t)sh.bc[0] - kFastBins / 2,
                           (int64_t)INT32_MIN);
  const uint32_t AB = (uint32_t)(int32_t)AB64;
  uint32_t nb = 0;
  auto bin = [&](int32_t xv) {
    const uint32_t d = (uint32_t)xv - AB;
    // samples outside the bins (d >= kFastBins as unsigned: above them, or
    // below them with the top bit set) go by one unsigned minimum to the
    // lane's own sink bin (no branch, and no two lanes of a warp collide
    // there)
    atomicAdd(&sh.hist[min(d, (uint32_t)(kFastBins + lane))], 1u);
    nb += d >> 31;
  };
  while (have) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      reinterpret_cast<int4 *>(buf + (h + u) * 128)[lane] = v[u];
      sx += (uint32_t)v[u].x + (uint32_t)v[u].y + (uint32_t)v[u].z +
            (uint32_t)v[u].w;
      mn32 = __vimin3_s32(mn32, __vimin3_s32(v[u].x, v[u].y, v[u].z), v[u].w);
      mx32 = __vimax3_s32(mx32, __vimax3_s32(v[u].x, v[u].y, v[u].z), v[u].w);
      if (binning) {
        bin(v[u].x);
        bin(v[u].y);
        bin(v[u].z);
        bin(v[u].w);
      }
    }
    h += 4;
    have = batch_ok(h);
    if (have) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
        v[u] = __ldg(reinterpret_cast<const int4 *>(x + (h + u) * 128) + lane);
    }
  }
  for (; h < 2 * g1; ++h) {
    const int b4 = h * 128 + 4 * lane;
    if (!DDSP_BC(b4 + 4 <= bufcap, kBcSpsBuf, b4)) continue;
    if (vec && b4 + 4 <= elen &&
        DDSP_BC(lo + b4 + 4 <= n, kBcSpsLoad, lo + b4)) {
      const int4 w4 = __ldg(reinterpret_cast<const int4 *>(x + b4));
      *reinterpret_cast<int4 *>(buf + b4) = w4;
      sx += (uint32_t)w4.x + (uint32_t)w4.y + (uint32_t)w4.z + (uint32_t)w4.w;
      if (b4 + 4 <= len) {
        mn32 = __vimin3_s32(mn32, __vimin3_s32(w4.x, w4.y, w4.z), w4.w);
        mx32 = __vimax3_s32(mx32, __vimax3_s32(w4.x, w4.y, w4.z), w4.w);
        if (binning) {
          bin(w4.x);
          bin(w4.y);
          bin(w4.z);
          bin(w4.w);
        }
      } else {
        const int32_t e4[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          take(b4 + e, e4[e]);
          if (binning && b4 + e < len) bin(e4[e]);
        }
      }
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = b4 + e;
        if (i < elen && DDSP_BC(lo + i < n, kBcSpsLoad, lo + i)) {
          const int32_t xv = __ldg(x + i);
          buf[i] = xv;
          sx += (uint32_t)xv;
          take(i, xv);
          if (binning && i < len) bin(xv);
        }
      }
    }
  }
  nb = __reduce_add_sync(0xffffffffu, nb);
  if (lane == 0) sh.nbw[warp] = nb;
  sx = __reduce_add_sync(0xffffffffu, sx);
  if (lane == 0) sh.wsx[run] = sx;
  mn32 = __reduce_min_sync(0xffffffffu, mn32);
  mx32 = __reduce_max_sync(0xffffffffu, mx32);
  hmn = __reduce_min_sync(0xffffffffu, hmn);
  hmx = __reduce_max_sync(0xffffffffu, hmx);
  if (lane == 0) {
    sh.wred[warp][0] = (uint32_t)mn32;
    sh.wred[warp][1] = (uint32_t)mx32;
    sh.hred[warp][0] = (uint32_t)hmn;
    sh.hred[warp][1] = (uint32_t)hmx;
  }
  __syncthreads();
  int64_t mn = INT32_MAX, mx = INT32_MIN, fmn, fmx;
  int64_t hn = INT32_MAX, hx = INT32_MIN;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    mn = min(mn, (int64_t)(int32_t)sh.wred[w][0]);
    mx = max(mx, (int64_t)(int32_t)sh.wred[w][1]);
    hn = min(hn, (int64_t)(int32_t)sh.hred[w][0]);
    hx = max(hx, (int64_t)(int32_t)sh.hred[w][1]);
  }
  fmn = min(mn, hn);    // everything loaded: window and look-ahead
  fmx = max(mx, hx);
  // (no barrier: wred and hred are written again only by select2's
  // fallback, after barriers every thread passes once it has read them)

  // ---- 2. median and MAD.  On the one-pass path the block finds the median,
  // then warps 0 and 1 (the lightest load and scan runs) search the MAD's
  // two ranks; the other warps wait at the barrier (the scan's chunk
  // statistics reuse the bins' space, so it cannot start earlier).  Either
  // part falls back to select2 when its ranks leave the bins.
  int64_t M2 = 0, MAD4 = 0;
  const bool range_ok = given || (mx - mn) < (int64_t)1 << 31;
  if (given) {
    M2 = m2_out[(int64_t)k * nwin + j];
    MAD4 = mad4_out[(int64_t)k * nwin + j];
  } else if (range_ok) {
    const int r1 = (len - 1) / 2, r2 = len / 2;
    const uint32_t base = (uint32_t)(int32_t)mn;
    uint32_t k1, k2, below = 0;
    // keys x - min in [0, 2^31)
    auto kx = [&](int i) { return (uint32_t)buf[i] - base; };
    // the bins' counts hold when every window sample lies within 2^31
    // of AB (below it: top bit set; from it up: clear)
    const bool fast = binning && mx - AB64 < ((int64_t)1 << 31) &&
                      AB64 - mn <= ((int64_t)1 << 31) &&
                      median_fast(AB64 - mn, r1, r2, sh, k1, k2, below);
    if (!fast)
      select2(kx, len, r1, r2, (uint32_t)(mx - mn), sh, k1, k2);
    M2 = 2 * mn + (int64_t)k1 + (int64_t)k2;
    bool mad_done = false;
    if (fast) {
      if (warp < 2) mad_fast_warp(AB64 - mn, below, k1, k2, r1, r2, sh);
      __syncthreads();
      const int64_t v1 = sh.bc[4], v2 = sh.bc[5];
      mad_done = v1 >= 0 && v2 >= 0;   // block-uniform
      MAD4 = v1 + v2;
    }
    if (!mad_done) {
      // |2x - M2| = |2(x - min) - (M2 - 2 min)|, both terms in [0, 2^32)
      const uint32_t m2r = (uint32_t)(M2 - 2 * mn);
      const uint64_t umax = (uint64_t)max(2 * mx - M2, M2 - 2 * mn);
      uint32_t u1, u2;
      select2(
          [&](int i) {
            const uint32_t t2 = 2u * ((uint32_t)buf[i] - base);
            return t2 >= m2r ? t2 - m2r : m2r - t2;
          },
          len, r1, r2, (uint32_t)umax, sh, u1, u2);
      MAD4 = (int64_t)u1 + (int64_t)u2;
    }
  } else if (tid == 0) {
    atomicExch(err, kErrRange);
  }

  // per-width FP32 scale 1/(2 sigma sqrt(w)) and integer screen thresholds
  // (set by warp 0, the lightest scan run, before its scan).
  // S/N >= thr  <=>  2 B_y - w*odd >= thr * 2 sigma sqrt(w); the screen
  // keeps a 4e-6 relative margin below that so FP32 rounding cannot hide a
  // candidate the FP32 S/N would accept.  Q2 (|2x - M2| <= 2 ybound + 1,
  // ybound the larger distance of floor(median) to the extremes of
  // everything loaded; that times elen + 1 below 2^30, so every prefix
  // value is below 2^30 in magnitude and the chunk bounds stay exact, and
  // times w_max below 2^22, so every numerator 2 B_y - w*odd converts
  // exactly): the prefix holds 2x - M2 and the threshold is on the
  // numerator itself; else on B_y.
  const int32_t mfloor = (int32_t)(M2 >> 1);  // floor(median)
  const int odd = (int)(M2 & 1);
  const int64_t ybound = max(fmx - (int64_t)mfloor, (int64_t)mfloor - fmn);
  const bool q2 = range_ok &&
                  (2 * ybound + 1) * (int64_t)(elen + 1) < ((int64_t)1 << 30) &&
                  (2 * ybound + 1) * (int64_t)wmax < ((int64_t)1 << 22);
  auto thresholds = [&](int64_t mad4) {
    if (lane < nw) {
      const float w = (float)widths[lane];
      // (a 32-bit conversion when MAD4 fits, the same rounding; the 64-bit
      // one runs on the FP64 pipe)
      const float mad4f = mad4 < ((int64_t)1 << 31)
                              ? __int2float_rn((int32_t)mad4)
                              : (float)mad4;
      const float two_sigma = kMadToSigma * mad4f * 0.5f;
      const float denom = two_sigma * sqrtf(w);
      sh.inv[lane] = mad4 > 0 ? 1.0f / denom : 0.0f;
      const float tnum = thr * denom * (1.0f - 4e-6f);
      const float t = q2 ? tnum : 0.5f * (tnum + (float)(widths[lane] * odd));
      int32_t tb;
      if (mad4 <= 0 || !(t < 2.0e9f)) tb = INT32_MAX;
      else if (t <= -2.0e9f) tb = INT32_MIN;
      else tb = (int32_t)floorf(t);
      sh.thr_by[lane] = tb;
      sh.wid[lane] = widths[lane];
    }
    if (lane == 0) {
      if (!given) {
        m2_out[(int64_t)k * nwin + j] = M2;
        mad4_out[(int64_t)k * nwin + j] = mad4;
      }
    }
  };
  if (warp == 0) thresholds(MAD4);
  // ---- 3. y (Q2: 2x - M2, else x - floor(median)) and its exclusive prefix
  // sum Q, in place: buf[p] = Q[p] = sum_{t < p} y[t] for p = 0 .. elen
  // (uint32, modular, so every difference Q[t + w] - Q[t] is exact).
  // Groups of 256 positions, a lane taking 8 consecutive ones (one chunk)
  // with two 16-byte shared loads, each warp a contiguous run of groups:
  // the runs' totals follow from the sums of x the load took, so one pass
  // scans with every warp's offset known, recording each lane's chunk
  // statistics on the way.  Statistics are kept only when every prefix
  // value fits in 30 bits in magnitude (the bound on |y| times (elen + 1)
  // below 2^30), where minima, maxima and their differences are exact.
  const int64_t ybnd = q2 ? 2 * ybound + 1 : ybound;
  const bool bounds = !DENSE && have_stats && range_ok && MAD4 > 0 &&
                     elen > 0 && ybnd * (int64_t)(elen + 1) < ((int64_t)1 << 30);
  {
    // y = x * ymul - ysub (mod 2^32)
    const uint32_t ymul = q2 ? 2u : 1u;
    const uint32_t ysub = q2 ? (uint32_t)M2 : (uint32_t)mfloor;
    // this run's offset: the totals of y over the runs before it, from the
    // sums of x the load took (a run holds the positions
    // [256 r gpw, 256 min(ngroups, (r + 1) gpw)), those below elen carry a
    // sample); every warp computes its own, so no barrier
    uint32_t carry = 0;
    if (lane < run) {
      const int r0 = lane * gpw * kGroup;
      const int r1 = min(ngroups, (lane + 1) * gpw) * kGroup;
      const int cnt = max(0, min(r1, elen) - r0);
      carry = sh.wsx[lane] * ymul - (uint32_t)cnt * ysub;
    }
    carry = __reduce_add_sync(0xffffffffu, carry);
    for (int g = g0; g < g1; ++g) {
      // this lane's 8 consecutive positions = one chunk of the statistics
      const int b8 = g * kGroup + kChunk * lane;
      // (a failed check leaves this lane's values out; the warp's scan
      // below still runs with all lanes)
      const bool in_buf = DDSP_BC(b8 + 8 <= bufcap, kBcSpsScan, b8);
      int4 va = make_int4(0, 0, 0, 0), vb = va;
      if (in_buf) {
        va = *reinterpret_cast<const int4 *>(buf + b8);
        vb = *reinterpret_cast<const int4 *>(buf + b8 + 4);
      }
      const int32_t xv[8] = {va.x, va.y, va.z, va.w, vb.x, vb.y, vb.z, vb.w};
      uint32_t y[8];
      if (b8 + 8 <= elen) {
#pragma unroll
        for (int e = 0; e < 8; ++e) y[e] = (uint32_t)xv[e] * ymul - ysub;
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e)
          y[e] = b8 + e < elen ? (uint32_t)xv[e] * ymul - ysub : 0u;
      }
      uint32_t ex[8];        // exclusive prefix inside the chunk
      ex[0] = 0u;
#pragma unroll
      for (int e = 1; e < 8; ++e) ex[e] = ex[e - 1] + y[e - 1];
      const uint32_t tot = ex[7] + y[7];
      const uint32_t inc = warp_incl_scan(tot, lane);
      const uint32_t pre = carry + inc - tot;
      if (in_buf) {
        *reinterpret_cast<uint4 *>(buf + b8) =
            make_uint4(pre + ex[0], pre + ex[1], pre + ex[2], pre + ex[3]);
        *reinterpret_cast<uint4 *>(buf + b8 + 4) =
            make_uint4(pre + ex[4], pre + ex[5], pre + ex[6], pre + ex[7]);
      }
      carry += __shfl_sync(0xffffffffu, inc, 31);
      if (bounds) {
        // Q = pre + ex, exact as int32 here (|Q| < 2^30); ex[0] = 0
        const int32_t e1 = (int32_t)ex[1], e2 = (int32_t)ex[2],
                      e3 = (int32_t)ex[3], e4 = (int32_t)ex[4],
                      e5 = (int32_t)ex[5], e6 = (int32_t)ex[6],
                      e7 = (int32_t)ex[7];
        const int32_t en = __vimin3_s32(__vimin3_s32(0, e1, e2),
                                        __vimin3_s32(e3, e4, e5),
                                        min(e6, e7));
        const int32_t exx = __vimax3_s32(__vimax3_s32(0, e1, e2),
                                         __vimax3_s32(e3, e4, e5),
                                         max(e6, e7));
        const int32_t ym = __vimax3_s32(
            __vimax3_s32((int32_t)y[0], (int32_t)y[1], (int32_t)y[2]),
            __vimax3_s32((int32_t)y[3], (int32_t)y[4], (int32_t)y[5]),
            max((int32_t)y[6], (int32_t)y[7]));
        const int c = b8 / kChunk;
        if (DDSP_BC(c < sps_chunk_cap(bufcap), kBcSpsStats, c)) {
          cmin[c] = (int32_t)pre + en;
          cmax[c] = (int32_t)pre + exx;
          ymax[c] = ym;
        }
      }
    }
    __syncthreads();
  }
  const uint32_t *Q = reinterpret_cast<const uint32_t *>(buf);

  // ---- 4. boxcars, S/N, candidates
  int32_t wv[kMaxWidths], tbv[kMaxWidths];
  float iv[kMaxWidths];
#pragma unroll
  for (int wi = 0; wi < kMaxWidths; ++wi) {
    const bool use = wi < nw;
    wv[wi] = use ? sh.wid[wi] : 0;
    tbv[wi] = use ? sh.thr_by[wi] : INT32_MAX;
    iv[wi] = use ? sh.inv[wi] : 0.0f;
  }
  // i + w <= n - lo also implies i + w <= elen, the last prefix index
  const int nv = (int)min(n - lo, (int64_t)elen);
  if (!DENSE && MAD4 <= 0)
    return;   // S/N 0 everywhere: no candidates (threshold > 0)
  bool pow2 = true;
#pragma unroll
  for (int wi = 0; wi < kMaxWidths; ++wi)
    pow2 = pow2 && (wi >= nw || wv[wi] == (1 << wi));
  // the warps' candidate stages: the histogram's space the chunk statistics
  // leave free (16-byte aligned), when it holds 32 records a warp
  uint32_t *stage = nullptr;
  int scap = 0;
  if (!DENSE) {
    const int used = stats_in_hist ? (int)((3 * ccap + 3) & ~3) : 0;
    const int per = ((kFastBins + 32 - used) / kWarps) & ~1;
    if (per >= 32) {
      stage = sh.hist + used;
      scap = per;
    }
  }
  const SweepArgs g{Q,     (int)bufcap, len,  nv,    nw,       odd,
                    mfloor, M2,         thr,  lo,    n,        nrep,
                    k,     wmax,        bounds, cmin, cmax,    ymax,
                    sh.wid, sh.inv,     stage, scap, cands, count, cap,
                    best_w, best_snr,   best_sum};
  // y prefix (not Q2) with |2 B_y - w*odd| < 2^22 for every width up to 32
  const bool n32 = !q2 && range_ok &&
                   (2 * ybound + 1) * 32 < ((int64_t)1 << 22);
  switch ((pow2 ? nw : 0) + (q2 ? 16 : (n32 && pow2 ? 32 : 0))) {
#define DDSP_SWEEP(N)                                     \
  case N:                                                 \
    sweep<DENSE, N, false>(g, wv, tbv, iv, bufcap);       \
    return;                                               \
  case N + 16:                                            \
    sweep<DENSE, N, true>(g, wv, tbv, iv, bufcap);        \
    return;                                               \
  case N + 32:                                            \
    sweep<DENSE, N, false, true>(g, wv, tbv, iv, bufcap); \
    return;
    DDSP_SWEEP(1) DDSP_SWEEP(2) DDSP_SWEEP(3) DDSP_SWEEP(4) DDSP_SWEEP(5)
    DDSP_SWEEP(6) DDSP_SWEEP(7) DDSP_SWEEP(8) DDSP_SWEEP(9) DDSP_SWEEP(10)
    DDSP_SWEEP(11)
#undef DDSP_SWEEP
    case 16:
      sweep<DENSE, 0, true>(g, wv, tbv, iv, bufcap);
      return;
    default:
      sweep<DENSE, 0, false>(g, wv, tbv, iv, bufcap);
  }
}

template <bool DENSE>
__global__ void __launch_bounds__(kSpsThreads, 4)
sps_kernel(const int32_t *__restrict__ series, int64_t n, int64_t L,
           int64_t nwin, const int32_t *__restrict__ widths, int nw, float thr,
           int64_t *__restrict__ m2_out, int64_t *__restrict__ mad4_out,
           ddsp_cand *__restrict__ cands, uint32_t *__restrict__ count,
           uint32_t cap, int32_t *__restrict__ best_w,
           float *__restrict__ best_snr, int32_t *__restrict__ best_sum,
           int32_t *__restrict__ err, int64_t bufcap) {
  sps_window<DENSE>(series, n, L, nwin, widths, nw, thr, m2_out, mad4_out,
                    cands, count, cap, best_w, best_snr, best_sum, err,
                    blockIdx.x, blockIdx.y, n, bufcap);
}

// Long mode, first pass: the exact median and MAD of each window straight
// from global memory (windows too long for shared memory): the window's
// minimum and maximum, then the histogram narrowing of select2 (2048 bins
// per pass over the window) for the two middle order statistics of
// x - min and of |2(x - min) - (m2 - 2 min)|; grid (window, DM trial).
__global__ void __launch_bounds__(kSpsThreads)
sps_long_stats_kernel(const int32_t *__restrict__ series, int64_t n, int64_t L,
                      int64_t nwin, int64_t *__restrict__ m2_out,
                      int64_t *__restrict__ mad4_out, int32_t *__restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SpsShared &sh = *reinterpret_cast<SpsShared *>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t j = blockIdx.x;
  const int k = blockIdx.y;
  const int64_t lo = (L <= 0) ? 0 : j * L;
  const int64_t hi = (L <= 0 || j == nwin - 1) ? n : (j + 1) * L;
  const int len = (int)(hi - lo);
  const int32_t *x = series + (int64_t)k * n + lo;
  int32_t mn32 = INT32_MAX, mx32 = INT32_MIN;
  for (int i = tid; i < len; i += kSpsThreads) {
    if (!DDSP_BC(lo + i < n, kBcSpsLoad, lo + i)) continue;
    const int32_t v = __ldg(x + i);
    mn32 = min(mn32, v);
    mx32 = max(mx32, v);
  }
  mn32 = __reduce_min_sync(0xffffffffu, mn32);
  mx32 = __reduce_max_sync(0xffffffffu, mx32);
  if (lane == 0) {
    sh.wred[warp][0] = (uint32_t)mn32;
    sh.wred[warp][1] = (uint32_t)mx32;
  }
  __syncthreads();
  int64_t mn = INT32_MAX, mx = INT32_MIN;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    mn = min(mn, (int64_t)(int32_t)sh.wred[w][0]);
    mx = max(mx, (int64_t)(int32_t)sh.wred[w][1]);
  }
  __syncthreads();
  int64_t M2 = 0, MAD4 = 0;
  if ((mx - mn) < (int64_t)1 << 31) {
    const int r1 = (len - 1) / 2, r2 = len / 2;
    const uint32_t base = (uint32_t)(int32_t)mn;
    uint32_t k1, k2, u1, u2;
    select2([&](int i) { return (uint32_t)__ldg(x + i) - base; }, len, r1, r2,
            (uint32_t)(mx - mn), sh, k1, k2);
    M2 = 2 * mn + (int64_t)k1 + (int64_t)k2;
    const uint32_t m2r = (uint32_t)(M2 - 2 * mn);
    const uint64_t umax = (uint64_t)max(2 * mx - M2, M2 - 2 * mn);
    select2(
        [&](int i) {
          const uint32_t t2 = 2u * ((uint32_t)__ldg(x + i) - base);
          return t2 >= m2r ? t2 - m2r : m2r - t2;
        },
        len, r1, r2, (uint32_t)umax, sh, u1, u2);
    MAD4 = (int64_t)u1 + (int64_t)u2;
  } else if (tid == 0) {
    atomicExch(err, kErrRange);
  }
  if (tid == 0) {
    m2_out[(int64_t)k * nwin + j] = M2;
    mad4_out[(int64_t)k * nwin + j] = MAD4;
  }
}

// Long mode, second pass: block (b, k) searches segment s of window j of DM
// trial k with that window's statistics; windows 0 .. nwin-2 (L samples)
// have segs_full segments each, the last window the rest.
template <bool DENSE>
__global__ void __launch_bounds__(kSpsThreads, 4)
sps_seg_kernel(const int32_t *__restrict__ series, int64_t n, int64_t L,
               int64_t nwin, const int32_t *__restrict__ widths, int nw,
               float thr, int64_t *__restrict__ m2_out,
               int64_t *__restrict__ mad4_out, ddsp_cand *__restrict__ cands,
               uint32_t *__restrict__ count, uint32_t cap,
               int32_t *__restrict__ best_w, float *__restrict__ best_snr,
               int32_t *__restrict__ best_sum, int32_t *__restrict__ err,
               int64_t bufcap, int64_t segs_full) {
  const int64_t bx = blockIdx.x;
  int64_t j, sg;
  if (nwin == 1) {
    j = 0;
    sg = bx;
  } else if (bx < (nwin - 1) * segs_full) {
    j = bx / segs_full;
    sg = bx - j * segs_full;
  } else {
    j = nwin - 1;
    sg = bx - (nwin - 1) * segs_full;
  }
  sps_window<DENSE>(series, n, L, nwin, widths, nw, thr, m2_out, mad4_out,
                    cands, count, cap, best_w, best_snr, best_sum, err, j,
                    blockIdx.y, n, bufcap, sg);
}

// Many beams in one launch: flattened block b -> the beam whose block0 is
// the largest <= b, then (DM trial, window) inside it.
__global__ void __launch_bounds__(kSpsThreads, 4)
sps_batch_kernel(const SpsBeam *__restrict__ beams, int nbeams, float thr,
                 int64_t bufcap) {
  const int64_t bid = blockIdx.x;
  int lo = 0, hi = nbeams - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (beams[mid].block0 <= bid) lo = mid; else hi = mid - 1;
  }
  const SpsBeam &b = beams[lo];
  const int64_t local = bid - b.block0;
  const int k = (int)(local / b.nwin);
  const int64_t j = local - (int64_t)k * b.nwin;
  sps_window<false>(b.series, b.n, b.L, b.nwin, b.widths, b.nw, thr, b.m2,
                    b.mad4, b.cands, b.count, b.cap, nullptr, nullptr,
                    nullptr, b.err, j, k, b.nrep, bufcap);
}

}  // namespace

int64_t sps_max_window_samples() { return kMaxWindowSamples; }

int64_t sps_bufcap(int64_t maxlen, int wmax) { return sps_buf_cap(maxlen, wmax); }

size_t sps_smem_bytes(int64_t maxlen, int wmax) {
  const int64_t cap = sps_buf_cap(maxlen, wmax);
  const int64_t ccap = sps_chunk_cap(cap);
  const bool separate = 3 * ccap > kFastBins && cap <= kStatsMaxCap;
  return kBufOff + 4 * (size_t)cap + (separate ? 12 * (size_t)ccap : 0);
}

// Largest dynamic shared memory a search launch asks for (the largest
// window the search accepts); the kernels are opted in to the device's
// limit once (smem_opt_in), shared by plan, batch, server and
// allocation-free launches and never lowered.
constexpr size_t kSpsMaxSmem =
    kBufOff + 4 * (size_t)(((kMaxWindowSamples + 1 + 255) / 256) * 256);

cudaError_t launch_sps_batch(const SpsBeam *d_beams, int nbeams,
                             int64_t total_blocks, float threshold,
                             size_t smem, int64_t bufcap, cudaStream_t s) {
  if (smem > kSpsMaxSmem) return cudaErrorInvalidValue;
  cudaError_t e = smem_opt_in(sps_batch_kernel);
  if (e != cudaSuccess) return e;
  sps_batch_kernel<<<(unsigned)total_blocks, kSpsThreads, smem, s>>>(
      d_beams, nbeams, threshold, bufcap);
  return cudaGetLastError();
}

cudaError_t launch_sps(const Plan &p, const int32_t *d_series,
                       int64_t nsamp_out, float threshold, bool dense,
                       int32_t *d_best_w, float *d_best_snr,
                       int32_t *d_best_sum, cudaStream_t s) {
  const int64_t L = p.norm_window;
  int64_t nwin = (L <= 0) ? 1 : max((int64_t)1, nsamp_out / L);
  int64_t maxlen = (L <= 0 || nwin == 1) ? nsamp_out
                                         : max(L, nsamp_out - (nwin - 1) * L);
  const int wmax = p.widths.back();
  if (maxlen + wmax > kMaxWindowSamples) {
    // long mode: statistics pass, then segments of kSeg start times
    cudaError_t e = cudaSuccess;
    sps_long_stats_kernel<<<dim3((unsigned)nwin, (unsigned)p.ndm), kSpsThreads,
                            kBufOff, s>>>(d_series, nsamp_out, L, nwin, p.d_m2,
                                          p.d_mad4, p.d_err);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t segs_full = L > 0 ? (L + kSeg - 1) / kSeg : 0;
    const int64_t last = nwin == 1 ? nsamp_out : nsamp_out - (nwin - 1) * L;
    const int64_t nblocks = (nwin - 1) * segs_full + (last + kSeg - 1) / kSeg;
    if (nblocks > 0x7fffffff) return cudaErrorInvalidValue;
    const size_t smem = sps_smem_bytes(kSeg, wmax);
    auto seg = dense ? sps_seg_kernel<true> : sps_seg_kernel<false>;
    if ((e = smem_opt_in(seg)) != cudaSuccess) return e;
    seg<<<dim3((unsigned)nblocks, (unsigned)p.ndm), kSpsThreads, smem, s>>>(
        d_series, nsamp_out, L, nwin, p.d_widths, p.nwidths, threshold, p.d_m2,
        p.d_mad4, p.d_cands, p.d_count, (uint32_t)p.cand_capacity, d_best_w,
        d_best_snr, d_best_sum, p.d_err, sps_buf_cap(kSeg, wmax), segs_full);
    return cudaGetLastError();
  }
  const size_t smem = sps_smem_bytes(maxlen, wmax);
  if (smem > kSpsMaxSmem) return cudaErrorInvalidValue;
  auto kern = dense ? sps_kernel<true> : sps_kernel<false>;
  cudaError_t e = smem_opt_in(kern);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)nwin, (unsigned)p.ndm);
  kern<<<grid, kSpsThreads, smem, s>>>(
      d_series, nsamp_out, L, nwin, p.d_widths, p.nwidths, threshold, p.d_m2,
      p.d_mad4, p.d_cands, p.d_count, (uint32_t)p.cand_capacity, d_best_w,
      d_best_snr, d_best_sum, p.d_err, sps_buf_cap(maxlen, wmax));
  return cudaGetLastError();
}

}  // namespace ddsp

// ===========================================================================
// Single-pulse search without any allocation.
//
// Some callers cannot call cudaMalloc: code that runs under a device memory
// budget fixed in advance, real-time loops where an allocation (which may
// synchronise the device) would break the latency budget, or hosts that
// hand this library pre-allocated buffers only.  For them the search's
// scratch -- the per-(DM trial, window) median/MAD statistics, the width
// table and the error word -- lives in one file-scope device array instead
// of a plan's workspace.  Every GPU that loads the library holds this array
// (a little over 4 MiB) until the process exits.
// ===========================================================================
namespace ddsp {
namespace {

constexpr int64_t kNoAllocMaxWindows = 262144;  // (DM trial, window) slots
constexpr size_t kNoAllocStatsBytes = (size_t)kNoAllocMaxWindows * 8;
// layout: m2[kNoAllocMaxWindows] | mad4[kNoAllocMaxWindows] | widths[16] |
//         error word
constexpr size_t kNoAllocWidthsOff = 2 * kNoAllocStatsBytes;
constexpr size_t kNoAllocErrOff = kNoAllocWidthsOff + 16 * sizeof(int32_t);
constexpr size_t kNoAllocBytes = kNoAllocErrOff + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
// device address of g_noalloc_scratch per device, found once per device
unsigned char *g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Everything a call must reset or refresh in the shared scratch, passed by
// value: the width table and the zeroed error word and counter.
struct NoAllocPrep {
  int32_t widths[kMaxWidths];
  int nw;
};

__global__ void noalloc_prep_kernel(NoAllocPrep a, int32_t *__restrict__ widths,
                                    int32_t *__restrict__ err,
                                    uint32_t *__restrict__ count) {
  const int t = threadIdx.x;
  if (t < a.nw) widths[t] = a.widths[t];
  if (t == 0) {
    *err = kErrNone;
    *count = 0u;
  }
}

// The scratch's device address on the current device (set-up on first use).
int noalloc_base(unsigned char **base) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices)
    return DDSP_E_CUDA;
  if (!g_noalloc_ptr[dev]) {
    // once per device, with that device current: the host-side name of the
    // array is only a stand-in, the kernel needs its device address
    unsigned char *ptr = nullptr;
    if (cudaGetSymbolAddress((void **)&ptr, g_noalloc_scratch) != cudaSuccess ||
        !ptr)
      return DDSP_E_CUDA;
    g_noalloc_ptr[dev] = ptr;
  }
  *base = g_noalloc_ptr[dev];
  return DDSP_OK;
}

}  // namespace
}  // namespace ddsp

extern "C" int ddsp_single_pulse_search_noalloc(
    const int32_t *d_series, int ndm, int64_t nsamp_out, const int *widths,
    int nwidths, int64_t norm_window, float threshold, ddsp_cand *d_cands,
    uint32_t cand_capacity, uint32_t *d_count, ddsp_stream_t stream) {
  using namespace ddsp;
  if (!d_series || !widths || !d_cands || !d_count || ndm <= 0 ||
      ndm > 65535 || nsamp_out <= 0 || nsamp_out > 0x7fffffffLL ||
      nwidths <= 0 || nwidths > kMaxWidths || norm_window < 0 ||
      cand_capacity == 0 || !(threshold > 0.0f) || !isfinite(threshold))
    return DDSP_E_INVALID_ARG;
  for (int i = 0; i < nwidths; ++i) {
    const int w = widths[i];
    if (w < 1 || w > 1024 || (w & (w - 1)) != 0) return DDSP_E_INVALID_ARG;
    if (i > 0 && w <= widths[i - 1]) return DDSP_E_INVALID_ARG;
  }
  const int64_t L = norm_window;
  const int64_t nwin = (L <= 0) ? 1 : max((int64_t)1, nsamp_out / L);
  const int64_t maxlen =
      (L <= 0 || nwin == 1) ? nsamp_out : max(L, nsamp_out - (nwin - 1) * L);
  const int wmax = widths[nwidths - 1];
  if (maxlen + wmax > kMaxWindowSamples) return DDSP_E_SHAPE;
  // the statistics of every (DM trial, window) must fit the static scratch
  if ((int64_t)ndm * nwin > kNoAllocMaxWindows) return DDSP_E_SHAPE;

  unsigned char *base = nullptr;
  const int brc = noalloc_base(&base);
  if (brc != DDSP_OK) return brc;
  int64_t *m2 = reinterpret_cast<int64_t *>(base);
  int64_t *mad4 = reinterpret_cast<int64_t *>(base + kNoAllocStatsBytes);
  int32_t *d_widths = reinterpret_cast<int32_t *>(base + kNoAllocWidthsOff);
  int32_t *d_err = reinterpret_cast<int32_t *>(base + kNoAllocErrOff);

  cudaStream_t s = (cudaStream_t)stream;
  const size_t smem = sps_smem_bytes(maxlen, wmax);
  auto kern = sps_kernel<false>;
  if (smem > kSpsMaxSmem || smem_opt_in(kern) != cudaSuccess)
    return DDSP_E_CUDA;
  // the array keeps the previous call's contents: one small launch resets
  // what must start at zero (the caller's counter and the error word) and
  // writes the widths, which travel as a kernel argument (no host copy)
  NoAllocPrep prep{};
  for (int i = 0; i < nwidths; ++i) prep.widths[i] = widths[i];
  prep.nw = nwidths;
  noalloc_prep_kernel<<<1, 32, 0, s>>>(prep, d_widths, d_err, d_count);
  if (cudaGetLastError() != cudaSuccess) return DDSP_E_CUDA;
  dim3 grid((unsigned)nwin, (unsigned)ndm);
  kern<<<grid, kSpsThreads, smem, s>>>(d_series, nsamp_out, L, nwin, d_widths,
                                       nwidths, threshold, m2, mad4, d_cands,
                                       d_count, cand_capacity, nullptr, nullptr,
                                       nullptr, d_err, sps_bufcap(maxlen, wmax));
  return cudaGetLastError() == cudaSuccess ? DDSP_OK : DDSP_E_CUDA;
}

extern "C" int ddsp_single_pulse_search_noalloc_check(ddsp_stream_t stream) {
  using namespace ddsp;
  unsigned char *base = nullptr;
  const int brc = noalloc_base(&base);
  if (brc != DDSP_OK) return brc;
  cudaStream_t s = (cudaStream_t)stream;
  int32_t *d_err = reinterpret_cast<int32_t *>(base + kNoAllocErrOff);
  int32_t v = kErrNone;
  if (cudaMemcpyAsync(&v, d_err, sizeof(v), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return DDSP_E_CUDA;
  if (v == kErrNone) return DDSP_OK;
  if (cudaMemsetAsync(d_err, 0, sizeof(int32_t), s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return DDSP_E_CUDA;
  return v == kErrRange ? DDSP_E_RANGE : DDSP_E_TIMEOUT;
}
