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
//      per add).  With two element buffers the relayout of chunk j+1
//      follows the accumulation of chunk j with one barrier;
//   3. every thread adds, for each of its RD DM trials and 4 elements, the
//      element at offset (delay - wbase) into SWAR accumulators, two
//      channels per step so the adds are 3-input:
//         acc_even += w & 0x00FF00FF   (bytes 0 and 2 in 16-bit lanes)
//         acc_odd  += w >> 8           (bytes 1..3 as b1 + 2^8 b2 + 2^16 b3)
//      Both stay exact for <= 256 channels (acc_odd <= 255*256*65793 <
//      2^32); at least every 256 channels they are unpacked into int32:
//         s0 = E & 0xFFFF, s2 = E >> 16, r = O - (s2 << 8),
//         s1 = r & 0xFFFF, s3 = r >> 16.
// Neighbouring DM trials of a tile have nearby delays, so one staged channel
// window serves all DT trials of the block.  The arithmetic is integer adds
// only; nothing here is a dense contraction, so no tensor cores are used.
#include <stdio.h>

#include <algorithm>

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

// Shared-memory layout of one block (bytes, all offsets 16-aligned):
//   [0, 32)                          up to four mbarriers, one per stage
//   rel_s[nbuf][cc*DT]               element-byte offsets of a staged chunk
//   raw[nbuf][cc][rawmax]            raw channel windows (bulk-copy targets)
//   elem[1|2][cc][elmax]             interleaved elements (uint32); with two
//                                    buffers the relayout of chunk j+1
//                                    follows the adds of chunk j with a
//                                    single barrier per chunk
struct SmemLayout {
  int rel_off, rel_stride, raw_off, elem_off, elem_stride, total;
  __host__ __device__ SmemLayout(int cc, int dt, int rawmax, int elmax,
                                 int nbuf, int nelem) {
    rel_off = 32;
    rel_stride = ((cc * dt * 4 + 15) / 16) * 16;
    raw_off = rel_off + nbuf * rel_stride;
    elem_off = raw_off + nbuf * cc * rawmax;
    elem_stride = cc * elmax * 4;
    total = elem_off + nelem * elem_stride;
  }
};

// Resident blocks per SM the register budget is set for: int32 totals held
// in registers (RTOT) cost 16*RD registers more per thread.
__host__ __device__ constexpr int dedisp_min_blocks(int rd, bool rtot) {
  return rtot ? (rd == 4 ? 2 : 3) : (rd == 4 ? 3 : 4);
}

template <int WT, int WD, int RD, bool DBUF, bool RTOT, typename T>
__global__ void __launch_bounds__(kThreads, dedisp_min_blocks(RD, RTOT))
dedisp_kernel(const T *__restrict__ cm, int64_t pitch, int nchan,
              int64_t nsamp_out, const int2 *__restrict__ desc,
              const int32_t *__restrict__ relb,
              const int32_t *__restrict__ rowmap, int32_t *__restrict__ out,
              int cc, int nbuf, int rawmax, int elmax, int32_t *err,
              long long timeout_cycles) {
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
  const SmemLayout L(cc, DT, rawmax, elmax, nbuf, DBUF ? 2 : 1);
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

  // Wait (bounded) for chunk j's copies and relayout it into its element
  // buffer, one warp per channel; only the elements the chunk's offsets can
  // reach are built.  Returns false if this thread's wait expired (it then
  // skips the relayout; the caller votes on the result at its barrier).
  auto stage_in = [&](int j) -> bool {
    const int st = j % nbuf;
    const int ncur = min(cc, nchan - j * cc);
    if (!mbar_wait(&bar[st], (uint32_t)((j / nbuf) & 1), timeout_cycles))
      return false;
    const int32_t *rel_s =
        reinterpret_cast<const int32_t *>(rel_base + st * L.rel_stride);
    const unsigned char *rb = raw + st * cc * rawmax;
    uint32_t *eb = reinterpret_cast<uint32_t *>(
        elem_base + (DBUF ? (j & 1) : 0) * L.elem_stride);
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
  int last_issued = min(nbuf - 2, nchunks - 1);  // same value in every thread

  // SWAR accumulators (uint8) and int32 totals.  With !RTOT (uint8 only)
  // the totals live in the output array: the owning thread adds each
  // <= 256-channel partial into its own outputs (the block's output tile
  // stays in L2), which frees 16*RD registers for more resident warps.
  constexpr bool kRegTot = RTOT || SPE != 4;
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
  bool first_flush = true;

  const int i0 = 32 * E * wt + lane;  // first element of this thread
  int failed_at = -1;
  int since = 0;  // channels in the SWAR accumulators since the last widen

  // prologue (two element buffers): chunk 0 into element buffer 0
  if (DBUF) {
    const bool ok = stage_in(0);
    if (__syncthreads_or(!ok)) failed_at = 0;
  }

  for (int j = 0; j < nchunks && failed_at < 0; ++j) {
    const int st = j % nbuf;
    const int ncur = min(cc, nchan - j * cc);
    // refill the raw stage the previous relayout consumed
    if (j + nbuf - 1 < nchunks) {
      if (warp == 0) {
        issue(j + nbuf - 1);
        load_desc(j + nbuf);
      }
      last_issued = j + nbuf - 1;
    }
    if (!DBUF) {
      const bool ok = stage_in(j);
      if (__syncthreads_or(!ok)) {
        failed_at = j;
        break;
      }
    }
    const int32_t *rel_s =
        reinterpret_cast<const int32_t *>(rel_base + st * L.rel_stride);

    // ---- accumulate chunk j from its element buffer, two channels at a
    // time: acc += (wa & M) + (wb & M) and acc += (wa >> 8) + (wb >> 8) map
    // to 3-input adds, which halves the add instructions per word
    const unsigned char *ebase =
        elem_base + (DBUF ? (j & 1) : 0) * L.elem_stride + 4 * i0;
    auto offsets = [&](int q, int (&rr)[RD]) {
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
    };
    int q = 0;
    for (; q + 1 < ncur; q += 2) {
      int ra[RD], rb[RD];
      offsets(q, ra);
      offsets(q + 1, rb);
      const unsigned char *ea = ebase + q * elmax * 4;
      const unsigned char *eb = ea + elmax * 4;
#pragma unroll
      for (int r = 0; r < RD; ++r) {
        const unsigned char *pa = ea + ra[r];
        const unsigned char *pb = eb + rb[r];
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const uint32_t wa = *reinterpret_cast<const uint32_t *>(pa + 128 * e);
          const uint32_t wb = *reinterpret_cast<const uint32_t *>(pb + 128 * e);
          if constexpr (SPE == 4) {
            accE[r][e] += (wa & 0x00FF00FFu) + (wb & 0x00FF00FFu);
            accO[r][e] += (wa >> 8) + (wb >> 8);
          } else {
            tot[r][e][0] += (int32_t)((wa & 0xFFFFu) + (wb & 0xFFFFu));
            tot[r][e][1] += (int32_t)((wa >> 16) + (wb >> 16));
          }
        }
      }
    }
    if (q < ncur) {
      int ra[RD];
      offsets(q, ra);
      const unsigned char *ea = ebase + q * elmax * 4;
#pragma unroll
      for (int r = 0; r < RD; ++r) {
        const unsigned char *pa = ea + ra[r];
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const uint32_t wa = *reinterpret_cast<const uint32_t *>(pa + 128 * e);
          if constexpr (SPE == 4) {
            accE[r][e] += wa & 0x00FF00FFu;
            accO[r][e] += wa >> 8;
          } else {
            tot[r][e][0] += (int32_t)(wa & 0xFFFFu);
            tot[r][e][1] += (int32_t)(wa >> 16);
          }
        }
      }
    }

    if constexpr (SPE == 4) {
      since += ncur;
      if (since + cc > 256 || j == nchunks - 1) {
        if constexpr (kRegTot) {
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
        } else {
#pragma unroll
          for (int r = 0; r < RD; ++r) {
            const int row = __ldg(rowmap + g * DT + RD * wd + r);
            int32_t *o = out + (int64_t)(row < 0 ? 0 : row) * nsamp_out;
#pragma unroll
            for (int e = 0; e < E; ++e) {
              uint32_t Ev = accE[r][e], O = accO[r][e];
              uint32_t s2 = Ev >> 16;
              uint32_t rem = O - (s2 << 8);
              int32_t part[4] = {(int32_t)(Ev & 0xFFFFu),
                                 (int32_t)(rem & 0xFFFFu), (int32_t)s2,
                                 (int32_t)(rem >> 16)};
#pragma unroll
              for (int m = 0; m < 4; ++m) {
                const int64_t t = T0 + i0 + 32 * e + (int64_t)m * S;
                if (row >= 0 && t < nsamp_out)
                  o[t] = first_flush ? part[m] : o[t] + part[m];
              }
              accE[r][e] = 0;
              accO[r][e] = 0;
            }
          }
          first_flush = false;
        }
        since = 0;
      }
    }

    if (DBUF) {
      // relayout chunk j + 1 into the other buffer; one barrier per chunk
      const bool ok = (j + 1 < nchunks) ? stage_in(j + 1) : true;
      if (__syncthreads_or(!ok)) failed_at = j + 1;
    } else {
      __syncthreads();  // the element buffer is rewritten next iteration
    }
  }

  if (failed_at >= 0) {
    if (tid == 0) {
      atomicExch(err, kErrTimeout);
      // let the copies still in flight land before the block retires, again
      // with a bounded wait per chunk
      for (int jj = failed_at; jj <= last_issued; ++jj)
        mbar_wait(&bar[jj % nbuf], (uint32_t)((jj / nbuf) & 1), timeout_cycles);
    }
    return;
  }

  // ---- store (without kRegTot the totals already sit in the output array)
  if constexpr (kRegTot) {
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
}

template <int WT, int WD, int RD, bool DBUF, bool RTOT, typename T>
cudaError_t launch_t(const Plan &p, const void *d_cm, int64_t pitch,
                     int64_t nsamp_out, int32_t *d_out, cudaStream_t s,
                     int rawmax, int elmax, size_t smem) {
  auto kern = dedisp_kernel<WT, WD, RD, DBUF, RTOT, T>;
  {
    cudaError_t e = smem_opt_in(kern);
    if (e != cudaSuccess) return e;
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
      p.d_err, timeout);
  return cudaGetLastError();
}

}  // namespace

// Interleaved elements per consumer thread: 4, except for the wide
// interleaved tile, where every thread holds 32 (DM trial, element) pairs.
int dedisp_elems_per_thread(const DedispTile &t) {
  const int wide = kTileInterleaved | kTileWide;
  return (t.flags & wide) == wide && t.rd > 0 ? 32 / t.rd : kElemPerThread;
}

// Elements per segment S (a time tile holds SPE segments).
int dedisp_segment(const DedispTile &t) {
  return 32 * dedisp_elems_per_thread(t) * t.wt;
}

// Time tile of a tile shape (samples per block).
static int time_tile_of(const DedispTile &t, int nbits) {
  return (nbits == 8 ? 4 : 2) * dedisp_segment(t);
}

void dedisp_buffer_sizes(const DedispTile &t, int span_max, int nbits,
                         int *rawmax, int *elmax);
static void buffer_sizes(const DedispTile &t, int span_max, int nbits,
                         int *rawmax, int *elmax) {
  dedisp_buffer_sizes(t, span_max, nbits, rawmax, elmax);
}

void dedisp_buffer_sizes(const DedispTile &t, int span_max, int nbits,
                         int *rawmax, int *elmax) {
  const int S = dedisp_segment(t);
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
  if (t.flags & kTileInterleaved)
    return dedisp_il_smem_bytes(t.chan_chunk, t.dm_tile(), elmax, t.nbuf);
  if (t.flags & kTileWarpSpecialized)
    return dedisp_ws_smem_bytes(t.chan_chunk, t.dm_tile(), rawmax, elmax,
                                t.nbuf);
  const bool dbuf = !(t.flags & kTileSingleElemBuffer);
  SmemLayout L(t.chan_chunk, t.dm_tile(), rawmax, elmax, t.nbuf, dbuf ? 2 : 1);
  return (size_t)L.total;
}

int dedisp_copy_bytes(const DedispTile &t, int span, int nbits) {
  if (t.flags & kTileInterleaved) {
    // elements 0 .. S + span - 1 of the window, whole 16-byte words
    const int S = dedisp_segment(t);
    return ((S + span + 3) & ~3) * 4;
  }
  const int TT = time_tile_of(t, nbits);
  return ((TT + span) * (nbits / 8) + 15) & ~15;
}

bool dedisp_tile_supported(const DedispTile &t, int nbits) {
  const bool wide = (t.flags & kTileWide) != 0;
  if (t.wt * t.wd != (wide ? 2 : 1) * (kThreads / 32)) return false;
  // instantiated variants (the dispatch list in launch_dedisperse): int32
  // totals in registers only with one element buffer; uint16 totals are
  // always in registers (the flag is implied)
  const int f = t.flags;
  if (f & kTileInterleaved) {
    if ((f & ~kTileWide) != kTileInterleaved) return false;
    if (t.rd != 4 && !(t.rd == 8 && nbits == 8)) return false;
    if (t.wd != 1 && t.wd != 2 && t.wd != 4) return false;
    if (nbits == 16 && t.rd == 8) return false;
    if (t.chan_chunk < 1 || t.chan_chunk > 32) return false;
    return t.nbuf >= 2 && t.nbuf <= dedisp_il_max_stages();
  }
  if (f & kTileWarpSpecialized) {
    if (f != kTileWarpSpecialized) return false;
    if (t.rd != 4 && !(t.rd == 8 && nbits == 8)) return false;
    if (t.wd != 1 && t.wd != 2 && t.wd != 4) return false;
    if (t.chan_chunk < 1 || t.chan_chunk > 32) return false;
    // each producer warp owns every other chunk and its own raw stages
    return t.nbuf == 2 || t.nbuf == 4;
  }
  if (f & ~(kTileSingleElemBuffer | kTileRegisterTotals)) return false;
  if (nbits == 8 && (f & kTileRegisterTotals) && !(f & kTileSingleElemBuffer))
    return false;
  if (nbits == 16 && (f & kTileRegisterTotals)) return false;
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
                              cudaStream_t s, int64_t ypitch) {
  int rawmax, elmax;
  buffer_sizes(p.tile, p.tab.span_max, p.nbits, &rawmax, &elmax);
  const size_t smem = dedisp_smem_bytes(p.tile, p.tab.span_max, p.nbits);
  if (p.tile.flags & kTileInterleaved) {
    // rebuild the interleaved rows from d_cm (null: p.d_il already holds
    // them); samples past nsamp_out + max_delay only reach discarded outputs
    if (d_cm) {
      const int64_t nvalid = std::min<int64_t>(pitch, nsamp_out + p.max_delay);
      cudaError_t e = launch_interleave(p, d_cm, pitch, nvalid, ypitch, s);
      if (e != cudaSuccess) return e;
    }
    return launch_dedisperse_il(p, ypitch, nsamp_out, d_out, s, elmax, smem);
  }
  if (p.tile.flags & kTileWarpSpecialized)
    return launch_dedisperse_ws(p, d_cm, pitch, nsamp_out, d_out, s, rawmax,
                                elmax, smem);
  const int wt = p.tile.wt, wd = p.tile.wd, rd = p.tile.rd;
  const int f = p.tile.flags;
  const bool dbuf = !(f & kTileSingleElemBuffer);
  const bool rtot = (f & kTileRegisterTotals) != 0;
#define DDSP_CASE(WT_, WD_, RD_, DB_, RT_, T_)                                \
  if (wt == WT_ && wd == WD_ && rd == RD_ && dbuf == DB_ && rtot == RT_)      \
    return launch_t<WT_, WD_, RD_, DB_, RT_, T_>(p, d_cm, pitch, nsamp_out,   \
                                                 d_out, s, rawmax, elmax,     \
                                                 smem);
#define DDSP_SHAPE8(WT_, WD_, RD_)                                            \
  DDSP_CASE(WT_, WD_, RD_, true, false, uint8_t)                              \
  DDSP_CASE(WT_, WD_, RD_, false, false, uint8_t)                             \
  DDSP_CASE(WT_, WD_, RD_, false, true, uint8_t)
#define DDSP_SHAPE16(WT_, WD_, RD_)                                           \
  DDSP_CASE(WT_, WD_, RD_, true, false, uint16_t)                             \
  DDSP_CASE(WT_, WD_, RD_, false, false, uint16_t)
  if (p.nbits == 8) {
    DDSP_SHAPE8(8, 1, 4)
    DDSP_SHAPE8(4, 2, 4)
    DDSP_SHAPE8(2, 4, 4)
    DDSP_SHAPE8(8, 1, 2)
    DDSP_SHAPE8(4, 2, 2)
    DDSP_SHAPE8(2, 4, 2)
  } else {
    DDSP_SHAPE16(8, 1, 4)
    DDSP_SHAPE16(4, 2, 4)
    DDSP_SHAPE16(2, 4, 4)
    DDSP_SHAPE16(8, 1, 2)
    DDSP_SHAPE16(4, 2, 2)
    DDSP_SHAPE16(2, 4, 2)
  }
#undef DDSP_SHAPE16
#undef DDSP_SHAPE8
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
