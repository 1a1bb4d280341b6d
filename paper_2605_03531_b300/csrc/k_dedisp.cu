// k_dedisp.cu -- brute-force incoherent dedispersion (Sec.3.2):
//   out[k][t] = sum_c x[c][t + d[k][c]],  exact in int32.
//
// Block = (DM tile of DT trials) x (time tile of TT output samples); the
// block loops over all channels in chunks of `cc`.  Per chunk:
//   1. one thread issues a 1-D TMA bulk copy (cp.async.bulk) per channel of
//      the raw window x[c][T0 + wbase(c) .. + TT + span(c)) into a shared
//      raw buffer (double-buffered; completion tracked by an mbarrier whose
//      waits are bounded);
//   2. all threads re-layout the raw window into "interleaved elements":
//      element i holds the samples i, i+S, i+2S, i+3S (uint8; two samples
//      i, i+S for uint16), S = TT/4.  A shifted read of element (i + delay)
//      then yields four output times at once whatever the delay's alignment,
//      so every 32-bit shared load feeds four adds (1 byte of shared traffic
//      per add);
//   3. every thread adds, for each of its 4 DM trials and 4 elements, the
//      element at offset (delay - wbase) into SWAR accumulators:
//         acc_even += w & 0x00FF00FF   (bytes 0 and 2 in 16-bit lanes)
//         acc_odd  += w >> 8           (bytes 1..3 as b1 + 2^8 b2 + 2^16 b3)
//      Both stay exact for <= 256 channels (acc_odd <= 255*256*65793 <
//      2^32); every 256 channels they are unpacked into int32 totals:
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

// Shared-memory layout of one block (bytes, all offsets 16-aligned):
//   [0, 16)                      two mbarriers
//   [16, 16 + 16*ceil(cc*DT/4))  relb_s: element-byte offsets of the chunk
//   raw[2][cc][rawmax]           raw channel windows (bulk-copy targets)
//   elem[cc][elmax]              interleaved elements (uint32)
struct SmemLayout {
  int rel_off, raw_off, elem_off, total;
  __host__ __device__ SmemLayout(int cc, int dt, int rawmax, int elmax) {
    rel_off = 16;
    int rel_bytes = ((cc * dt * 4 + 15) / 16) * 16;
    raw_off = rel_off + rel_bytes;
    elem_off = raw_off + 2 * cc * rawmax;
    total = elem_off + cc * elmax * 4;
  }
};

template <int WT, int WD, typename T>
__global__ void __launch_bounds__(kThreads, 2)
dedisp_kernel(const T *__restrict__ cm, int64_t pitch, int nchan,
              int64_t nsamp_out, const int32_t *__restrict__ wbase,
              const int32_t *__restrict__ relb,
              const int32_t *__restrict__ rowmap, int32_t *__restrict__ out,
              int cc, int rawmax, int elmax, int32_t *err,
              long long timeout_cycles) {
  constexpr int SPE = 4 / sizeof(T);               // samples per element
  constexpr int S = 32 * kElemPerThread * WT;      // elements per segment
  constexpr int TT = SPE * S;                      // samples per time tile
  constexpr int DT = kDmPerThread * WD;            // DM trials per tile

  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wt = warp % WT, wd = warp / WT;
  const int g = blockIdx.x;
  const int64_t T0 = (int64_t)blockIdx.y * TT;
  const SmemLayout L(cc, DT, rawmax, elmax);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  int32_t *rel_s = reinterpret_cast<int32_t *>(smem + L.rel_off);
  unsigned char *raw = smem + L.raw_off;
  uint32_t *elem = reinterpret_cast<uint32_t *>(smem + L.elem_off);

  const int nchunks = (nchan + cc - 1) / cc;
  const int32_t *wb_g = wbase + (int64_t)g * nchan;
  const int32_t *rel_g = relb + (int64_t)g * nchan * DT;

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();

  // One thread stages chunk j into raw buffer (j & 1).
  auto issue = [&](int j) {
    const int c0 = j * cc;
    const int ncur = min(cc, nchan - c0);
    uint32_t total = 0;
    for (int q = 0; q < ncur; ++q) {
      int span = rel_g[(int64_t)(c0 + q) * DT + DT - 1] / 4;
      total += ((TT + span) * (int)sizeof(T) + 15) & ~15;
    }
    uint64_t *b = &bar[j & 1];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(b, total);
    unsigned char *dst = raw + (j & 1) * cc * rawmax;
    for (int q = 0; q < ncur; ++q) {
      const int c = c0 + q;
      int span = rel_g[(int64_t)c * DT + DT - 1] / 4;
      uint32_t nb = ((TT + span) * (int)sizeof(T) + 15) & ~15;
      const T *src = cm + (int64_t)c * pitch + T0 + wb_g[c];
      bulk_g2s(dst + q * rawmax, src, nb, b);
    }
  };

  if (tid == 0) issue(0);

  // SWAR accumulators (uint8) or direct int32 sums (uint16).
  uint32_t accE[kDmPerThread][kElemPerThread];
  uint32_t accO[kDmPerThread][kElemPerThread];
  int32_t tot[kDmPerThread][kElemPerThread][SPE];
#pragma unroll
  for (int r = 0; r < kDmPerThread; ++r)
#pragma unroll
    for (int e = 0; e < kElemPerThread; ++e) {
      accE[r][e] = 0;
      accO[r][e] = 0;
#pragma unroll
      for (int m = 0; m < SPE; ++m) tot[r][e][m] = 0;
    }

  const int i0 = 32 * kElemPerThread * wt + lane;  // first element of thread
  int failed_at = -1;

  for (int j = 0; j < nchunks; ++j) {
    const int buf = j & 1;
    const int c0 = j * cc;
    if (tid == 0 && j + 1 < nchunks) issue(j + 1);
    bool ok = mbar_wait(&bar[buf], (uint32_t)((j >> 1) & 1), timeout_cycles);
    if (__syncthreads_or(!ok)) {
      failed_at = j;
      break;
    }
    // ---- relayout raw -> interleaved elements; stage the chunk's offsets
    for (int q = tid; q < cc * DT; q += kThreads) {
      int c = c0 + q / DT;
      rel_s[q] = (c < nchan) ? rel_g[(int64_t)c * DT + (q % DT)] : 0;
    }
    const unsigned char *rb = raw + buf * cc * rawmax;
    for (int q = 0; q < cc; ++q) {
      const bool valid = (c0 + q) < nchan;
      const unsigned char *rq = rb + q * rawmax;
      uint32_t *eq = elem + q * elmax;
      if constexpr (SPE == 4) {
        for (int i4 = tid; i4 < elmax / 4; i4 += kThreads) {
          uint4 o = make_uint4(0, 0, 0, 0);
          if (valid) {
            const unsigned char *p = rq + 4 * i4;
            uint32_t r0 = *reinterpret_cast<const uint32_t *>(p);
            uint32_t r1 = *reinterpret_cast<const uint32_t *>(p + S);
            uint32_t r2 = *reinterpret_cast<const uint32_t *>(p + 2 * S);
            uint32_t r3 = *reinterpret_cast<const uint32_t *>(p + 3 * S);
            uint32_t t0 = __byte_perm(r0, r1, 0x5140);
            uint32_t t1 = __byte_perm(r0, r1, 0x7362);
            uint32_t t2 = __byte_perm(r2, r3, 0x5140);
            uint32_t t3 = __byte_perm(r2, r3, 0x7362);
            o.x = __byte_perm(t0, t2, 0x5410);
            o.y = __byte_perm(t0, t2, 0x7632);
            o.z = __byte_perm(t1, t3, 0x5410);
            o.w = __byte_perm(t1, t3, 0x7632);
          }
          *reinterpret_cast<uint4 *>(eq + 4 * i4) = o;
        }
      } else {
        for (int i2 = tid; i2 < elmax / 2; i2 += kThreads) {
          uint2 o = make_uint2(0, 0);
          if (valid) {
            const unsigned char *p = rq + 4 * i2;
            uint32_t w0 = *reinterpret_cast<const uint32_t *>(p);
            uint32_t w1 = *reinterpret_cast<const uint32_t *>(p + 2 * S);
            o.x = __byte_perm(w0, w1, 0x5410);
            o.y = __byte_perm(w0, w1, 0x7632);
          }
          *reinterpret_cast<uint2 *>(eq + 2 * i2) = o;
        }
      }
    }
    __syncthreads();

    // ---- accumulate
    const unsigned char *ebase =
        reinterpret_cast<const unsigned char *>(elem) + 4 * i0;
#pragma unroll 2
    for (int q = 0; q < cc; ++q) {
      const int4 ro = *reinterpret_cast<const int4 *>(rel_s + q * DT +
                                                      kDmPerThread * wd);
      const int rr[4] = {ro.x, ro.y, ro.z, ro.w};
      const unsigned char *eq = ebase + q * elmax * 4;
#pragma unroll
      for (int r = 0; r < kDmPerThread; ++r) {
        const unsigned char *p = eq + rr[r];
#pragma unroll
        for (int e = 0; e < kElemPerThread; ++e) {
          uint32_t w = *reinterpret_cast<const uint32_t *>(p + 128 * e);
          if constexpr (SPE == 4) {
            accE[r][e] += w & 0x00FF00FFu;
            accO[r][e] += w >> 8;
          } else {
            tot[r][e][0] += (int32_t)(w & 0xFFFFu);
            tot[r][e][1] += (int32_t)(w >> 16);
          }
        }
      }
    }

    if constexpr (SPE == 4) {
      const int cend = c0 + cc;
      if ((cend & 255) == 0 || j == nchunks - 1) {
#pragma unroll
        for (int r = 0; r < kDmPerThread; ++r)
#pragma unroll
          for (int e = 0; e < kElemPerThread; ++e) {
            uint32_t E = accE[r][e], O = accO[r][e];
            uint32_t s2 = E >> 16;
            uint32_t rem = O - (s2 << 8);
            tot[r][e][0] += (int32_t)(E & 0xFFFFu);
            tot[r][e][1] += (int32_t)(rem & 0xFFFFu);
            tot[r][e][2] += (int32_t)s2;
            tot[r][e][3] += (int32_t)(rem >> 16);
            accE[r][e] = 0;
            accO[r][e] = 0;
          }
      }
    }
    __syncthreads();
  }

  if (failed_at >= 0) {
    if (tid == 0) {
      atomicExch(err, kErrTimeout);
      // let the copies still in flight (chunks failed_at and failed_at + 1)
      // land before the block retires, again with a bounded wait
      const int j = failed_at;
      mbar_wait(&bar[j & 1], (uint32_t)((j >> 1) & 1), timeout_cycles);
      if (j + 1 < nchunks)
        mbar_wait(&bar[(j + 1) & 1], (uint32_t)(((j + 1) >> 1) & 1),
                  timeout_cycles);
    }
    return;
  }

  // ---- store
#pragma unroll
  for (int r = 0; r < kDmPerThread; ++r) {
    const int row = rowmap[g * DT + kDmPerThread * wd + r];
    if (row < 0) continue;
    int32_t *o = out + (int64_t)row * nsamp_out;
#pragma unroll
    for (int e = 0; e < kElemPerThread; ++e)
#pragma unroll
      for (int m = 0; m < SPE; ++m) {
        const int64_t t = T0 + i0 + 32 * e + (int64_t)m * S;
        if (t < nsamp_out) o[t] = tot[r][e][m];
      }
  }
}

template <int WT, int WD, typename T>
cudaError_t launch_t(const Plan &p, const void *d_cm, int64_t pitch,
                     int64_t nsamp_out, int32_t *d_out, cudaStream_t s,
                     int rawmax, int elmax, size_t smem) {
  auto kern = dedisp_kernel<WT, WD, T>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(
        kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  constexpr int SPE = 4 / sizeof(T);
  constexpr int TT = SPE * 32 * kElemPerThread * WT;
  dim3 grid((unsigned)p.tab.n_dm_tiles,
            (unsigned)((nsamp_out + TT - 1) / TT));
  const long long timeout = 4000000000LL;  // ~2 s of SM clock
  kern<<<grid, kThreads, smem, s>>>(
      static_cast<const T *>(d_cm), pitch, p.nchan, nsamp_out, p.tab.d_wbase,
      p.tab.d_relb, p.tab.d_rowmap, d_out, p.tile.chan_chunk, rawmax, elmax,
      p.d_err, timeout);
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
  SmemLayout L(t.chan_chunk, t.dm_tile(), rawmax, elmax);
  return (size_t)L.total;
}

cudaError_t launch_dedisperse(const Plan &p, const void *d_cm, int64_t pitch,
                              int64_t nsamp_out, int32_t *d_out,
                              cudaStream_t s) {
  int rawmax, elmax;
  buffer_sizes(p.tile, p.tab.span_max, p.nbits, &rawmax, &elmax);
  const size_t smem = dedisp_smem_bytes(p.tile, p.tab.span_max, p.nbits);
  const int wt = p.tile.wt, wd = p.tile.wd;
#define DDSP_CASE(WT_, WD_)                                                  \
  if (wt == WT_ && wd == WD_)                                                \
    return p.nbits == 8                                                      \
               ? launch_t<WT_, WD_, uint8_t>(p, d_cm, pitch, nsamp_out,      \
                                             d_out, s, rawmax, elmax, smem)  \
               : launch_t<WT_, WD_, uint16_t>(p, d_cm, pitch, nsamp_out,     \
                                              d_out, s, rawmax, elmax, smem);
  DDSP_CASE(8, 1)
  DDSP_CASE(4, 2)
  DDSP_CASE(2, 4)
#undef DDSP_CASE
  return cudaErrorInvalidValue;
}

int dedisp_time_tile(const DedispTile &t, int nbits) {
  return time_tile_of(t, nbits);
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
