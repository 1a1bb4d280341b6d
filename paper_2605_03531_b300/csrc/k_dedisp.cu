// k_dedisp.cu -- brute-force incoherent dedispersion (Sec.3.2):
//   out[k][t] = sum_c x[c][t + d[k][c]],  exact in int32.
//
// Block = (DM tile of DT trials) x (time tile of TT output samples); the
// block loops over all channels in chunks of `cc`.  Per chunk:
//   1. warp 0 issues one 1-D TMA bulk copy (cp.async.bulk) per channel, one
//      lane per channel, of the raw window x[c][T0 + wbase(c) .. + TT +
//      span(c)), plus one copy of the chunk's delay offsets, into a shared
//      stage; `nbuf` stages keep up to nbuf-1 chunks in flight; completion
//      is tracked by one mbarrier per stage whose waits are bounded;
//   2. all warps re-layout the raw window into "interleaved elements":
//      element i holds the samples i, i+S, i+2S, i+3S (uint8; two samples
//      i, i+S for uint16), S = TT/4.  A shifted read of element (i + delay)
//      then yields four output times at once whatever the delay's alignment,
//      so every 32-bit shared load feeds four adds (1 byte of shared traffic
//      per add).  The element buffer is double-buffered: the relayout of
//      chunk j+1 follows the accumulation of chunk j with one barrier;
//   3. every thread adds, for each of its RD DM trials and 4 elements, the
//      element at offset (delay - wbase) into SWAR accumulators:
//         acc_even += w & 0x00FF00FF   (bytes 0 and 2 in 16-bit lanes)
//         acc_odd  += w >> 8           (bytes 1..3 as b1 + 2^8 b2 + 2^16 b3,
//                                       as mad.hi on the FMA pipe)
//      Both stay exact for <= 256 channels (acc_odd <= 255*256*65793 <
//      2^32); at least every 256 channels they are unpacked into int32:
//         s0 = E & 0xFFFF, s2 = E >> 16, r = O - (s2 << 8),
//         s1 = r & 0xFFFF, s3 = r >> 16.
// Neighbouring DM trials of a tile have nearby delays, so one staged channel
// window serves all DT trials of the block.  The arithmetic is integer adds
// only; nothing here is a dense contraction, so no tensor cores are used.
#include <stdio.h>

#include "internal.h"

namespace ddsp {
namespace {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile(
      "mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
          smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src,
                                         uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Bounded wait on an mbarrier phase: false if `limit` cycles pass first.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          long long limit) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}

// acc += w >> 8 on the FMA pipe: mad.hi(w, 2^24, acc).  `k24` is 2^24 held
// in a register so the multiply is not turned back into an ALU shift.
__device__ __forceinline__ uint32_t add_hi(uint32_t acc, uint32_t w,
                                           uint32_t k24) {
  uint32_t r;
  asm("mad.hi.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(w), "r"(k24), "r"(acc));
  return r;
}

// Shared-memory layout of one block (bytes, all offsets 16-aligned):
//   [0, 32)                          up to four mbarriers, one per stage
//   rel_s[nbuf][cc*DT]               element-byte offsets of a staged chunk
//   raw[nbuf][cc][rawmax]            raw channel windows (bulk-copy targets)
//   elem[2][cc][elmax]               interleaved elements (uint32)
struct SmemLayout {
  int rel_off, rel_stride, raw_off, elem_off, elem_stride, total;
  __host__ __device__ SmemLayout(int cc, int dt, int rawmax, int elmax,
                                 int nbuf) {
    rel_off = 32;
    rel_stride = ((cc * dt * 4 + 15) / 16) * 16;
    raw_off = rel_off + nbuf * rel_stride;
    elem_off = raw_off + nbuf * cc * rawmax;
    elem_stride = cc * elmax * 4;
    total = elem_off + 2 * elem_stride;
  }
};

template <int WT, int WD, int RD, typename T>
__global__ void __launch_bounds__(kThreads, RD == 4 ? 2 : 3)
dedisp_kernel(const T *__restrict__ cm, int64_t pitch, int nchan,
              int64_t nsamp_out, const int2 *__restrict__ desc,
              const int32_t *__restrict__ relb,
              const int32_t *__restrict__ rowmap, int32_t *__restrict__ out,
              int cc, int nbuf, int rawmax, int elmax, uint32_t k24,
              int32_t *err, long long timeout_cycles) {
  constexpr int SPE = 4 / sizeof(T);               // samples per element
  constexpr int E = kElemPerThread;
  constexpr int S = 32 * E * WT;                   // elements per segment
  constexpr int TT = SPE * S;                      // samples per time tile
  constexpr int DT = RD * WD;                      // DM trials per tile
  constexpr int kWarps = kThreads / 32;

  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wt = warp % WT, wd = warp / WT;
  const int g = blockIdx.x;
  const int64_t T0 = (int64_t)blockIdx.y * TT;
  const SmemLayout L(cc, DT, rawmax, elmax, nbuf);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  unsigned char *rel_base = smem + L.rel_off;
  unsigned char *raw = smem + L.raw_off;
  unsigned char *elem_base = smem + L.elem_off;

  const int nchunks = (nchan + cc - 1) / cc;
  const int2 *desc_g = desc + (int64_t)g * nchan;
  const int32_t *rel_g = relb + (int64_t)g * nchan * DT;

  if (tid == 0) {
    for (int b = 0; b < nbuf; ++b) mbar_init(&bar[b], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();

  // ---- producer: warp 0, one lane per channel of a chunk.  `nd` holds the
  // copy descriptor {window start, bytes} of the lane's channel of the next
  // chunk to issue; it is loaded one issue ahead so its latency is hidden.
  int2 nd = make_int2(0, 0);
  auto load_desc = [&](int j) {
    const int c = j * cc + lane;
    if (lane < cc && j < nchunks && c < nchan) nd = __ldg(desc_g + c);
  };
  auto issue = [&](int j) {
    const int c0 = j * cc;
    const int ncur = min(cc, nchan - c0);
    const bool v = lane < ncur;
    const uint32_t nb = v ? (uint32_t)nd.y : 0u;
    const uint32_t relbytes = (uint32_t)(ncur * DT * 4);
    const uint32_t total = __reduce_add_sync(0xffffffffu, nb) + relbytes;
    const int st = j % nbuf;
    if (lane == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(&bar[st], total);
    }
    __syncwarp();
    if (v)
      bulk_g2s(raw + (st * cc + lane) * rawmax,
               cm + (int64_t)(c0 + lane) * pitch + T0 + nd.x, nb, &bar[st]);
    if (lane == 0)
      bulk_g2s(rel_base + st * L.rel_stride, rel_g + (int64_t)c0 * DT,
               relbytes, &bar[st]);
  };

  // Wait for chunk j's copies, then relayout it into element buffer j & 1,
  // one warp per channel; only the elements the chunk's offsets can reach
  // are built.  Returns false (uniformly) if the bounded wait expired.
  auto stage_in = [&](int j) -> bool {
    const int st = j % nbuf;
    const int ncur = min(cc, nchan - j * cc);
    bool ok = mbar_wait(&bar[st], (uint32_t)((j / nbuf) & 1), timeout_cycles);
    if (__syncthreads_or(!ok)) return false;
    const int32_t *rel_s =
        reinterpret_cast<const int32_t *>(rel_base + st * L.rel_stride);
    const unsigned char *rb = raw + st * cc * rawmax;
    uint32_t *eb =
        reinterpret_cast<uint32_t *>(elem_base + (j & 1) * L.elem_stride);
    for (int q = warp; q < ncur; q += kWarps) {
      const unsigned char *rq = rb + q * rawmax;
      uint32_t *eq = eb + q * elmax;
      const int span = rel_s[q * DT + DT - 1] >> 2;
      if constexpr (SPE == 4) {
        const int nq = (S + span + 3) >> 2;
        for (int i4 = lane; i4 < nq; i4 += 32) {
          const unsigned char *p = rq + 4 * i4;
          uint32_t r0 = *reinterpret_cast<const uint32_t *>(p);
          uint32_t r1 = *reinterpret_cast<const uint32_t *>(p + S);
          uint32_t r2 = *reinterpret_cast<const uint32_t *>(p + 2 * S);
          uint32_t r3 = *reinterpret_cast<const uint32_t *>(p + 3 * S);
          uint32_t t0 = __byte_perm(r0, r1, 0x5140);
          uint32_t t1 = __byte_perm(r0, r1, 0x7362);
          uint32_t t2 = __byte_perm(r2, r3, 0x5140);
          uint32_t t3 = __byte_perm(r2, r3, 0x7362);
          uint4 o;
          o.x = __byte_perm(t0, t2, 0x5410);
          o.y = __byte_perm(t0, t2, 0x7632);
          o.z = __byte_perm(t1, t3, 0x5410);
          o.w = __byte_perm(t1, t3, 0x7632);
          *reinterpret_cast<uint4 *>(eq + 4 * i4) = o;
        }
      } else {
        const int nq = (S + span + 1) >> 1;
        for (int i2 = lane; i2 < nq; i2 += 32) {
          const unsigned char *p = rq + 4 * i2;
          uint32_t w0 = *reinterpret_cast<const uint32_t *>(p);
          uint32_t w1 = *reinterpret_cast<const uint32_t *>(p + 2 * S);
          uint2 o;
          o.x = __byte_perm(w0, w1, 0x5410);
          o.y = __byte_perm(w0, w1, 0x7632);
          *reinterpret_cast<uint2 *>(eq + 2 * i2) = o;
        }
      }
    }
    return true;
  };

  if (warp == 0) {
    for (int j = 0; j < nbuf - 1 && j < nchunks; ++j) {
      load_desc(j);
      issue(j);
    }
    load_desc(nbuf - 1);
  }

  // SWAR accumulators (uint8) or direct int32 sums (uint16).
  uint32_t accE[RD][E];
  uint32_t accO[RD][E];
  int32_t tot[RD][E][SPE];
#pragma unroll
  for (int r = 0; r < RD; ++r)
#pragma unroll
    for (int e = 0; e < E; ++e) {
      accE[r][e] = 0;
      accO[r][e] = 0;
#pragma unroll
      for (int m = 0; m < SPE; ++m) tot[r][e][m] = 0;
    }

  const int i0 = 32 * E * wt + lane;  // first element of this thread
  int failed_at = -1;
  int since = 0;  // channels in the SWAR accumulators since the last widen

  // prologue: chunk 0 into element buffer 0
  if (!stage_in(0)) failed_at = 0;
  __syncthreads();

  for (int j = 0; j < nchunks && failed_at < 0; ++j) {
    const int st = j % nbuf;
    const int ncur = min(cc, nchan - j * cc);
    // refill the raw stage the previous relayout consumed
    if (warp == 0 && j + nbuf - 1 < nchunks) {
      issue(j + nbuf - 1);
      load_desc(j + nbuf);
    }
    const int32_t *rel_s =
        reinterpret_cast<const int32_t *>(rel_base + st * L.rel_stride);

    // ---- accumulate chunk j from element buffer j & 1
    const unsigned char *ebase = elem_base + (j & 1) * L.elem_stride + 4 * i0;
#pragma unroll 2
    for (int q = 0; q < ncur; ++q) {
      int rr[RD];
      if constexpr (RD == 4) {
        const int4 ro =
            *reinterpret_cast<const int4 *>(rel_s + q * DT + RD * wd);
        rr[0] = ro.x;
        rr[1] = ro.y;
        rr[2] = ro.z;
        rr[3] = ro.w;
      } else {
        const int2 ro =
            *reinterpret_cast<const int2 *>(rel_s + q * DT + RD * wd);
        rr[0] = ro.x;
        rr[1] = ro.y;
      }
      const unsigned char *eq = ebase + q * elmax * 4;
#pragma unroll
      for (int r = 0; r < RD; ++r) {
        const unsigned char *p = eq + rr[r];
#pragma unroll
        for (int e = 0; e < E; ++e) {
          uint32_t w = *reinterpret_cast<const uint32_t *>(p + 128 * e);
          if constexpr (SPE == 4) {
            accE[r][e] += w & 0x00FF00FFu;
            accO[r][e] = add_hi(accO[r][e], w, k24);
          } else {
            tot[r][e][0] += (int32_t)(w & 0xFFFFu);
            tot[r][e][1] += (int32_t)(w >> 16);
          }
        }
      }
    }

    if constexpr (SPE == 4) {
      since += ncur;
      if (since + cc > 256 || j == nchunks - 1) {
#pragma unroll
        for (int r = 0; r < RD; ++r)
#pragma unroll
          for (int e = 0; e < E; ++e) {
            uint32_t Ev = accE[r][e], O = accO[r][e];
            uint32_t s2 = Ev >> 16;
            uint32_t rem = O - (s2 << 8);
            tot[r][e][0] += (int32_t)(Ev & 0xFFFFu);
            tot[r][e][1] += (int32_t)(rem & 0xFFFFu);
            tot[r][e][2] += (int32_t)s2;
            tot[r][e][3] += (int32_t)(rem >> 16);
            accE[r][e] = 0;
            accO[r][e] = 0;
          }
        since = 0;
      }
    }

    // ---- relayout chunk j + 1 into the other element buffer
    if (j + 1 < nchunks && !stage_in(j + 1)) failed_at = j + 1;
    __syncthreads();
  }

  if (failed_at >= 0) {
    if (tid == 0) {
      atomicExch(err, kErrTimeout);
      // let the copies still in flight land before the block retires, again
      // with a bounded wait per chunk
      const int last = min(failed_at + nbuf - 2, nchunks - 1);
      for (int jj = failed_at; jj <= last; ++jj)
        mbar_wait(&bar[jj % nbuf], (uint32_t)((jj / nbuf) & 1), timeout_cycles);
    }
    return;
  }

  // ---- store
#pragma unroll
  for (int r = 0; r < RD; ++r) {
    const int row = rowmap[g * DT + RD * wd + r];
    if (row < 0) continue;
    int32_t *o = out + (int64_t)row * nsamp_out;
#pragma unroll
    for (int e = 0; e < E; ++e)
#pragma unroll
      for (int m = 0; m < SPE; ++m) {
        const int64_t t = T0 + i0 + 32 * e + (int64_t)m * S;
        if (t < nsamp_out) o[t] = tot[r][e][m];
      }
  }
}

template <int WT, int WD, int RD, typename T>
cudaError_t launch_t(const Plan &p, const void *d_cm, int64_t pitch,
                     int64_t nsamp_out, int32_t *d_out, cudaStream_t s,
                     int rawmax, int elmax, size_t smem) {
  auto kern = dedisp_kernel<WT, WD, RD, T>;
  static size_t attr_bytes = 0;
  if (smem > attr_bytes) {
    cudaError_t e = cudaFuncSetAttribute(
        kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_bytes = smem;
  }
  constexpr int SPE = 4 / sizeof(T);
  constexpr int TT = SPE * 32 * kElemPerThread * WT;
  dim3 grid((unsigned)p.tab.n_dm_tiles,
            (unsigned)((nsamp_out + TT - 1) / TT));
  const long long timeout = 4000000000LL;  // ~2 s of SM clock
  kern<<<grid, kThreads, smem, s>>>(
      static_cast<const T *>(d_cm), pitch, p.nchan, nsamp_out,
      reinterpret_cast<const int2 *>(p.tab.d_desc), p.tab.d_relb,
      p.tab.d_rowmap, d_out, p.tile.chan_chunk, p.tile.nbuf, rawmax, elmax,
      1u << 24, p.d_err, timeout);
  return cudaGetLastError();
}

}  // namespace

// Time tile of a tile shape (samples per block).
static int time_tile_of(const DedispTile &t, int nbits) {
  return (nbits == 8 ? 4 : 2) * 32 * kElemPerThread * t.wt;
}

static void buffer_sizes(const DedispTile &t, int span_max, int nbits,
                         int *rawmax, int *elmax) {
  const int S = 32 * kElemPerThread * t.wt;
  const int TT = time_tile_of(t, nbits);
  const int bps = nbits / 8;
  *elmax = ((S + span_max + 4) + 3) & ~3;
  // the relayout of element i reads raw samples up to i + (SPE-1)*S
  int need = (*elmax + (TT - S)) * bps;
  int copy = ((TT + span_max) * bps + 15) & ~15;
  int r = need > copy ? need : copy;
  *rawmax = (r + 15) & ~15;
}

size_t dedisp_smem_bytes(const DedispTile &t, int span_max, int nbits) {
  int rawmax, elmax;
  buffer_sizes(t, span_max, nbits, &rawmax, &elmax);
  SmemLayout L(t.chan_chunk, t.dm_tile(), rawmax, elmax, t.nbuf);
  return (size_t)L.total;
}

int dedisp_copy_bytes(const DedispTile &t, int span, int nbits) {
  const int TT = time_tile_of(t, nbits);
  return ((TT + span) * (nbits / 8) + 15) & ~15;
}

bool dedisp_tile_supported(const DedispTile &t) {
  if (t.wt * t.wd != kThreads / 32) return false;
  if (t.rd != 2 && t.rd != 4) return false;
  if (t.wd != 1 && t.wd != 2 && t.wd != 4) return false;
  if (t.chan_chunk < 1 || t.chan_chunk > 32) return false;
  return t.nbuf >= 2 && t.nbuf <= 4;
}

int dedisp_time_tile(const DedispTile &t, int nbits) {
  return time_tile_of(t, nbits);
}

cudaError_t launch_dedisperse(const Plan &p, const void *d_cm, int64_t pitch,
                              int64_t nsamp_out, int32_t *d_out,
                              cudaStream_t s) {
  int rawmax, elmax;
  buffer_sizes(p.tile, p.tab.span_max, p.nbits, &rawmax, &elmax);
  const size_t smem = dedisp_smem_bytes(p.tile, p.tab.span_max, p.nbits);
  const int wt = p.tile.wt, wd = p.tile.wd, rd = p.tile.rd;
#define DDSP_CASE(WT_, WD_, RD_)                                             \
  if (wt == WT_ && wd == WD_ && rd == RD_)                                   \
    return p.nbits == 8                                                      \
               ? launch_t<WT_, WD_, RD_, uint8_t>(p, d_cm, pitch, nsamp_out, \
                                                  d_out, s, rawmax, elmax,   \
                                                  smem)                      \
               : launch_t<WT_, WD_, RD_, uint16_t>(p, d_cm, pitch,           \
                                                   nsamp_out, d_out, s,      \
                                                   rawmax, elmax, smem);
  DDSP_CASE(8, 1, 4)
  DDSP_CASE(4, 2, 4)
  DDSP_CASE(2, 4, 4)
  DDSP_CASE(8, 1, 2)
  DDSP_CASE(4, 2, 2)
  DDSP_CASE(2, 4, 2)
#undef DDSP_CASE
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Direct kernel: one thread per (DM trial, 4 consecutive output samples),
// channel samples read straight from the channel-major rows through the
// read-only cache.  No staging and no on-chip footprint limit, so it serves
// DM grids whose delay spread inside a tile would not fit in shared memory.
namespace {
template <typename T>
__global__ void __launch_bounds__(256)
dedisp_direct_kernel(const T *__restrict__ cm, int64_t pitch, int nchan,
                     int64_t nsamp_out, const int32_t *__restrict__ delays,
                     int32_t *__restrict__ out) {
  const int k = blockIdx.y;
  const int64_t t0 = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  if (t0 >= nsamp_out) return;
  const int32_t *dk = delays + (int64_t)k * nchan;
  int32_t acc[4] = {0, 0, 0, 0};
  for (int c = 0; c < nchan; ++c) {
    const T *row = cm + (int64_t)c * pitch + t0 + __ldg(dk + c);
#pragma unroll
    for (int m = 0; m < 4; ++m) acc[m] += (int32_t)__ldg(row + m);
  }
  int32_t *o = out + (int64_t)k * nsamp_out;
#pragma unroll
  for (int m = 0; m < 4; ++m)
    if (t0 + m < nsamp_out) o[t0 + m] = acc[m];
}
}  // namespace

cudaError_t launch_dedisperse_direct(const Plan &p, const void *d_cm,
                                     int64_t pitch, int64_t nsamp_out,
                                     int32_t *d_out, cudaStream_t s) {
  dim3 grid((unsigned)((nsamp_out + 1023) / 1024), (unsigned)p.ndm);
  if (p.nbits == 8)
    dedisp_direct_kernel<uint8_t><<<grid, 256, 0, s>>>(
        static_cast<const uint8_t *>(d_cm), pitch, p.nchan, nsamp_out,
        p.d_delays, d_out);
  else
    dedisp_direct_kernel<uint16_t><<<grid, 256, 0, s>>>(
        static_cast<const uint16_t *>(d_cm), pitch, p.nchan, nsamp_out,
        p.d_delays, d_out);
  return cudaGetLastError();
}

}  // namespace ddsp
