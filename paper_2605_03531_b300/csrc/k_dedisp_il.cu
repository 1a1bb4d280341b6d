// k_dedisp_il.cu -- brute-force dedispersion (Sec.3.2) from pre-interleaved
// channel rows: out[k][t] = sum_c x[c][t + d[k][c]], exact in int32.
//
// The consumer arithmetic (ws_item.cuh) reads one 32-bit element per DM
// trial that holds the samples of SPE output times S apart: element i of a
// time tile = {x[i], x[i+S], x[i+2S], x[i+3S]} (uint8) or {x[i], x[i+S]}
// (uint16).  That element does not depend on the tile: it is Y[i] of the
// channel's interleaved row Y, which one streaming pass (interleave_kernel)
// writes once per block of data.  The dedispersion kernel then stages its
// windows of Y with 1-D TMA bulk copies straight into the element stages,
// with no on-chip relayout: one producer warp only issues copies, and the
// stages form an nst-deep ring (full / empty mbarriers) in front of the
// consumer warps.  Y costs 4 bytes per sample in HBM (uint8; 2 for uint16)
// and its windows are re-read from L2 across DM tiles, which is cheap next
// to the shared-memory reads and writes the relayout took per element.
//
// Every wait is bounded; a role that gives up records a timeout, the
// producer drains its copies in flight (bounded), and the block returns.
#include "host.h"
#include "ws_item.cuh"

namespace ddsp {
namespace {

constexpr int kIlMaxStages = 8;
constexpr int kIlBarBytes = 128;   // full[8], empty[8]

// Shared memory: [0, 128) mbarriers, then nst stages of
//   rel[cc][DT] int32 (element-byte offsets, 16-byte padded)
//   elem[cc][elmax] uint32 (the channels' windows of Y)
struct IlLayout {
  int rel_stride, stage_stride, total;
  __host__ __device__ IlLayout(int cc, int dt, int elmax, int nst) {
    rel_stride = ((cc * dt * 4 + 15) / 16) * 16;
    stage_stride = rel_stride + cc * elmax * 4;
    total = kIlBarBytes + nst * stage_stride;
  }
};

struct IlArgs {
  const uint32_t *y;      // [nchan][ypitch] interleaved rows
  int64_t ypitch;         // elements
  int64_t nsamp_out;
  int64_t out_pitch;
  const int2 *desc;       // [n_dm_tiles][nchan] {window start, bytes}
  const int32_t *relb;    // [n_dm_tiles][nchan][DT] element-byte offsets
  const int32_t *rowmap;  // [n_dm_tiles*DT] output row or -1
  int32_t *out;           // [ndm][out_pitch]
  int nchan, cc, elmax, nst;
  uint32_t one;           // 1: the multiplier of the FMA-pipe adds (a
                          // kernel argument, so the compiler cannot fold it)
  int nz;                 // > 0: blockIdx.z picks rows and output from z[]
  int withhold;           // >= 0: the producer stops before this chunk
                          // (failure-detection test; -1 in normal use)
  IlRows z[kIlMaxRows];   // (same tables, same shape: e.g. beam-blocks)
};

// Y[c][i] for i in [0, ypitch): byte (uint8) or half (uint16) m holds
// x[c][i + m S] if that index is below nvalid, else 0.  One thread builds 4
// consecutive elements from SPE aligned loads (a 4x4 byte transpose for
// uint8) and stores them as one 16-byte word.  (Four such groups a thread,
// for more loads in flight, ran 10 % slower: fewer threads.)
// With ring > 0 the rows are rings: logical sample b sits at (t0 + b) %
// ring; t0, ring, S and i are multiples of 4, so a 4-sample group never
// straddles the wrap.
template <typename T>
__global__ void __launch_bounds__(256)
interleave_kernel(const T *__restrict__ cm, int64_t pitch, int64_t nvalid,
                  int S, uint32_t *__restrict__ y, int64_t ypitch,
                  int64_t ring, int64_t t0) {
  constexpr int SPE = 4 / sizeof(T);
  const int c = blockIdx.y;
  const int64_t i = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  if (i >= ypitch || !DDSP_BC(i + 4 <= ypitch, kBcIntlvOut, i)) return;
  const T *x = cm + (int64_t)c * pitch;
  // ring position of logical sample b: a window never spans more than one
  // wrap (t0 < ring, b < ring), so one compare and subtraction does it (a
  // 64-bit remainder per load cost 18 % of the kernel's time); the
  // remainder stays as a fallback
  auto at = [&](int64_t b) {
    if (ring <= 0) return b;
    int64_t q = t0 + b;
    if (q >= ring) q -= ring;
    return q < ring ? q : q % ring;
  };
  uint4 o;
  if constexpr (SPE == 4) {
    uint32_t w[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int64_t b = i + (int64_t)m * S;
      if (b + 4 <= nvalid) {
        const int64_t a = at(b);
        w[m] = DDSP_BC(a >= 0 && a + 4 <= pitch, kBcIntlvIn, a)
                   ? __ldg(reinterpret_cast<const uint32_t *>(x + a))
                   : 0u;
      } else {
        uint32_t v = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (b + k < nvalid) v |= (uint32_t)x[at(b + k)] << (8 * k);
        w[m] = v;
      }
    }
    o = transpose4x4(w[0], w[1], w[2], w[3]);
  } else {
    uint32_t h[2][4];
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      const int64_t b = i + (int64_t)m * S;
      if (b + 4 <= nvalid) {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(x + at(b)));
        h[m][0] = v.x & 0xFFFFu;
        h[m][1] = v.x >> 16;
        h[m][2] = v.y & 0xFFFFu;
        h[m][3] = v.y >> 16;
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) h[m][k] = b + k < nvalid ? x[at(b + k)] : 0u;
      }
    }
    o.x = h[0][0] | (h[1][0] << 16);
    o.y = h[0][1] | (h[1][1] << 16);
    o.z = h[0][2] | (h[1][2] << 16);
    o.w = h[0][3] | (h[1][3] << 16);
  }
  *reinterpret_cast<uint4 *>(y + (int64_t)c * ypitch + i) = o;
}

// The uint8 interleave with 16-byte loads, for rows, segment length S,
// ring length and ring start that are multiples of 16 (a 16-sample group
// then never straddles the wrap): a thread builds 16 consecutive elements
// from four 16-byte loads (rows i + m S), four 4x4 byte transposes, four
// 16-byte stores.
__global__ void __launch_bounds__(256)
interleave16_u8_kernel(const uint8_t *__restrict__ cm, int64_t pitch,
                       int64_t nvalid, int S, uint32_t *__restrict__ y,
                       int64_t ypitch, int64_t ring, int64_t t0) {
  const int c = blockIdx.y;
  const int64_t i = 16 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  if (i >= ypitch) return;
  const uint8_t *x = cm + (int64_t)c * pitch;
  auto at = [&](int64_t b) {
    if (ring <= 0) return b;
    int64_t q = t0 + b;
    if (q >= ring) q -= ring;
    return q < ring ? q : q % ring;
  };
  uint4 w[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int64_t b = i + (int64_t)m * S;
    if (b + 16 <= nvalid) {
      const int64_t a = at(b);
      w[m] = DDSP_BC(a >= 0 && a + 16 <= pitch, kBcIntlvIn, a)
                 ? __ldg(reinterpret_cast<const uint4 *>(x + a))
                 : make_uint4(0u, 0u, 0u, 0u);
    } else {
      uint32_t v[4] = {0u, 0u, 0u, 0u};
#pragma unroll
      for (int k = 0; k < 16; ++k)
        if (b + k < nvalid) v[k >> 2] |= (uint32_t)x[at(b + k)] << (8 * (k & 3));
      w[m] = make_uint4(v[0], v[1], v[2], v[3]);
    }
  }
  uint32_t *yr = y + (int64_t)c * ypitch + i;
  const uint4 q0 = transpose4x4(w[0].x, w[1].x, w[2].x, w[3].x);
  const uint4 q1 = transpose4x4(w[0].y, w[1].y, w[2].y, w[3].y);
  const uint4 q2 = transpose4x4(w[0].z, w[1].z, w[2].z, w[3].z);
  const uint4 q3 = transpose4x4(w[0].w, w[1].w, w[2].w, w[3].w);
  if (i + 4 <= ypitch && DDSP_BC(true, kBcIntlvOut, i))
    reinterpret_cast<uint4 *>(yr)[0] = q0;
  if (i + 8 <= ypitch && DDSP_BC(true, kBcIntlvOut, i + 4))
    reinterpret_cast<uint4 *>(yr)[1] = q1;
  if (i + 12 <= ypitch && DDSP_BC(true, kBcIntlvOut, i + 8))
    reinterpret_cast<uint4 *>(yr)[2] = q2;
  if (i + 16 <= ypitch && DDSP_BC(true, kBcIntlvOut, i + 12))
    reinterpret_cast<uint4 *>(yr)[3] = q3;
}

// Time-major uint8 spectra (nchan % 16 == 0) straight to interleaved rows:
// a block takes 64 elements x 128 channels, i.e. the four 64-sample x
// 128-channel tiles of input rows i0 + m S (m < 4), loaded as 16-byte
// vectors along channels.  A thread turns each 4x4 byte block (4 samples x
// 4 channels) of every tile into 4 channel words with byte permutes, then
// the 4 tiles' words of one channel into 4 elements (a second 4x4
// transpose), stored as one 16-byte word along time.
constexpr int kIlTS = 64;              // elements per block
constexpr int kIlTC = 128;             // channels per block
constexpr int kIlPW = kIlTC / 4 + 1;   // tile row pitch in words (skew)

__global__ void __launch_bounds__(256)
unpack_interleave_u8_kernel(const uint8_t *__restrict__ in, int64_t nsamp_in,
                            int nchan, int S, uint32_t *__restrict__ y,
                            int64_t ypitch, int time_on_y) {
  __shared__ uint32_t tile[4][kIlTS * kIlPW];
  const int tid = threadIdx.x;
  // time_on_y: blockIdx.x is the channel slice, so the slices of one time
  // range run together and write neighbouring parts of every row (10 %
  // faster than the slices one after another)
  const int64_t i0 = (int64_t)(time_on_y ? blockIdx.y : blockIdx.x) * kIlTS;
  const int c0 = (time_on_y ? blockIdx.x : blockIdx.y) * kIlTC;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int idx = tid + 256 * k;     // 64 rows x 8 vectors
      const int row = idx >> 3, q = idx & 7;
      const int64_t smp = i0 + row + (int64_t)m * S;
      const int c = c0 + 16 * q;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (smp < nsamp_in && c < nchan &&
          DDSP_BC(c + 16 <= nchan, kBcStageIn, c))
        v = __ldg(reinterpret_cast<const uint4 *>(in + smp * nchan + c));
      uint32_t *dst = tile[m] + row * kIlPW + 4 * q;
      dst[0] = v.x;
      dst[1] = v.y;
      dst[2] = v.z;
      dst[3] = v.w;
    }
  }
  __syncthreads();
  const int lane = tid & 31, w = tid >> 5;
  const int sq = lane & 15;              // elements 4 sq .. 4 sq + 3
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const int cq = (lane >> 4) + 2 * w + 16 * it;   // channels 4 cq ..
    uint32_t cw[4][4];                   // [m][channel j]: 4 samples
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const uint32_t *src = tile[m] + (4 * sq) * kIlPW + cq;
      const uint4 o = transpose4x4(src[0], src[kIlPW], src[2 * kIlPW],
                                   src[3 * kIlPW]);
      cw[m][0] = o.x;
      cw[m][1] = o.y;
      cw[m][2] = o.z;
      cw[m][3] = o.w;
    }
    const int64_t i = i0 + 4 * sq;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + 4 * cq + j;
      if (c < nchan && i < ypitch &&
          DDSP_BC(i + 4 <= ypitch, kBcStageOut, i))
        *reinterpret_cast<uint4 *>(y + (int64_t)c * ypitch + i) =
            transpose4x4(cw[0][j], cw[1][j], cw[2][j], cw[3][j]);
    }
  }
}

// One block per (DM tile, time tile): warp NC is the producer, warps
// 0..NC-1 the consumers (WT along time x WD along DM).  NC = 8: two blocks
// per SM; NC = 16 (wide tile): one block per SM, twice the time tile and
// the chunk, so each chunk's synchronisation and each window's delay span
// are spread over twice the adds.  Either way an SM sub-partition holds 5
// warps, whose 16K registers allow 96 a thread (the bound below).
template <int WT, int WD, int RD, int E, typename T>
__global__ void __launch_bounds__(WT * WD == 16 ? 640 : 32 * (WT * WD + 1),
                                  WT * WD == 16 ? 1 : 2)
dedisp_il_kernel(IlArgs a, int32_t *err, long long timeout_cycles) {
  constexpr int SPE = 4 / sizeof(T);
  constexpr int S = 32 * E * WT;     // elements per segment
  constexpr int TT = SPE * S;        // output samples per tile
  constexpr int DT = RD * WD;
  constexpr int NC = WT * WD;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t *full = reinterpret_cast<uint64_t *>(smem);
  uint64_t *empty = full + kIlMaxStages;
  const int cc = a.cc, elmax = a.elmax, nst = a.nst, nchan = a.nchan;
  const IlLayout L(cc, DT, elmax, nst);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = blockIdx.x;
  const int64_t T0 = (int64_t)blockIdx.y * TT;
  const int nchunks = (nchan + cc - 1) / cc;
  unsigned char *stages = smem + kIlBarBytes;
  const uint32_t *yrows = a.nz > 0 ? a.z[blockIdx.z].y : a.y;
  int32_t *out = a.nz > 0 ? a.z[blockIdx.z].out : a.out;

  if (tid == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NC);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();

  if (warp == NC) {
    // ============================= producer =============================
    const int2 *desc_g = a.desc + (int64_t)g * nchan;
    const int32_t *rel_g = a.relb + (int64_t)g * nchan * DT;
    // copy descriptors of channels [base, base + 32) and the 32 after them,
    // lane l holding channel base + l: a chunk (cc <= 32) spans at most the
    // two, and each batch is loaded one batch ahead of its use, so no chunk
    // waits on a global load
    auto ld_desc = [&](int c) {
      return c < nchan ? __ldg(desc_g + c) : make_int2(0, 0);
    };
    int base = 0;
    int2 dcur = ld_desc(lane), dnext = ld_desc(32 + lane);
    int j = 0;
    // ring position of chunk j: stage st, pass (j / nst) parity ph
    int st = 0;
    uint32_t ph = 0;
    bool withheld = false;
    for (; j < nchunks; ++j) {
      if (j == a.withhold) {   // test switch: this chunk is never staged
        withheld = true;
        break;
      }
      // the stage's previous chunk (j - nst) has been consumed (the warp
      // gives up as a whole if any lane's wait ran out)
      if (!__all_sync(0xffffffffu,
                      mbar_wait(&empty[st], ph ^ 1u, timeout_cycles)))
        break;
      const int c0 = j * cc;
      const int ncur = min(cc, nchan - c0);
      const bool v = lane < ncur;
      const int off = c0 - base + lane;          // < 64
      const int src = off & 31;
      const int2 da = make_int2(__shfl_sync(0xffffffffu, dcur.x, src),
                                __shfl_sync(0xffffffffu, dcur.y, src));
      const int2 db = make_int2(__shfl_sync(0xffffffffu, dnext.x, src),
                                __shfl_sync(0xffffffffu, dnext.y, src));
      const int2 d = off < 32 ? da : db;
      if (c0 + ncur >= base + 32) {    // the next chunk starts past dcur
        base += 32;
        dcur = dnext;
        dnext = ld_desc(base + 32 + lane);
      }
      uint32_t nb = v ? (uint32_t)d.y : 0u;
      const uint32_t relbytes = (uint32_t)(ncur * DT * 4);
#ifdef DDSP_BOUNDS_CHECK
      // the window [T0 + start, + nb/4) inside the row, the copy inside the
      // channel's slot of the stage; a failing copy is left out (its bytes
      // too, so the stage still completes)
      if (v && !(DDSP_BC(T0 + d.x >= 0 && T0 + d.x + nb / 4 <= a.ypitch,
                         kBcIlSrc, T0 + d.x) &&
                 DDSP_BC(nb <= (uint32_t)elmax * 4u && (nb & 15u) == 0,
                         kBcIlDst, nb)))
        nb = 0u;
      DDSP_BC(relbytes <= (uint32_t)L.rel_stride, kBcIlRel, relbytes);
#endif
      const uint32_t total = __reduce_add_sync(0xffffffffu, nb) + relbytes;
      unsigned char *sb = stages + st * L.stage_stride;
      if (lane == 0) mbar_expect_tx(&full[st], total);
      __syncwarp();
      if (v && nb > 0u)
        bulk_g2s(sb + L.rel_stride + lane * elmax * 4,
                 yrows + (int64_t)(c0 + lane) * a.ypitch + T0 + d.x, nb,
                 &full[st]);
      if (lane == 0)
        bulk_g2s(sb, rel_g + (int64_t)c0 * DT, relbytes, &full[st]);
      if (++st == nst) {
        st = 0;
        ph ^= 1u;
      }
    }
    if (j < nchunks) {
      // gave up (or withheld a chunk): record it and let the copies in
      // flight (chunks j - nst .. j - 1) land before the block's shared
      // memory goes away; these waits keep the default bound whatever the
      // hand-off bound is, as the copies were issued and will land
      if (lane == 0) {
        if (!withheld) atomicExch(err, kErrTimeout);
        for (int jj = max(0, j - nst); jj < j; ++jj)
          mbar_wait(&full[jj % nst], (uint32_t)((jj / nst) & 1),
                    kDefaultWaitCycles);
      }
    }
    return;
  }

  // ============================= consumers ==============================
  const int wt = warp % WT, wd = warp / WT;
  const int i0 = 32 * E * wt + lane;  // first element of this thread
  const uint32_t one = a.one;
  WsAcc<RD, SPE, E> acc;
  acc.zero();
  bool first_flush = true;
  int since = 0;
  int st = 0;
  uint32_t ph = 0;
  for (int j = 0; j < nchunks; ++j) {
    const int ncur = min(cc, nchan - j * cc);
    if (!__all_sync(0xffffffffu, mbar_wait(&full[st], ph, timeout_cycles))) {
      if (lane == 0) atomicExch(err, kErrTimeout);
      return;
    }
    const unsigned char *sb = stages + st * L.stage_stride;
    ws_accumulate(acc, reinterpret_cast<const int32_t *>(sb) + RD * wd, DT,
                  sb + L.rel_stride + 4 * i0, elmax, ncur, one, i0);
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[st]);
    if (++st == nst) {
      st = 0;
      ph ^= 1u;
    }
    if constexpr (SPE == 4) {
      since += ncur;
      if (since + cc > 256 || j == nchunks - 1) {
        ws_flush(acc, a.rowmap + g * DT + RD * wd, out, a.out_pitch,
                 T0 + i0, S, a.nsamp_out, first_flush);
        first_flush = false;
        since = 0;
      }
    }
  }
  if constexpr (SPE != 4)
    ws_store_totals(acc, a.rowmap + g * DT + RD * wd, out, a.out_pitch,
                    T0 + i0, S, a.nsamp_out);
}

template <int WT, int WD, int RD, int E, typename T>
cudaError_t launch_il_t(const IlLaunch &p, int64_t ypitch, int64_t nsamp_out,
                        int32_t *d_out, cudaStream_t s, int elmax,
                        size_t smem, int64_t out_pitch, const IlRows *rows,
                        int nrows) {
  auto kern = dedisp_il_kernel<WT, WD, RD, E, T>;
  {
    cudaError_t e = smem_opt_in(kern);
    // the largest shared-memory carveout, so two blocks fit beside each other
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kern,
                               cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  constexpr int SPE = 4 / sizeof(T);
  constexpr int TT = SPE * 32 * E * WT;
  const int ntt = (int)((nsamp_out + TT - 1) / TT);
  IlArgs a{};
  a.y = static_cast<const uint32_t *>(p.d_il);
  a.ypitch = ypitch;
  a.nsamp_out = nsamp_out;
  a.out_pitch = out_pitch > 0 ? out_pitch : nsamp_out;
  a.desc = reinterpret_cast<const int2 *>(p.tab->d_desc);
  a.relb = p.tab->d_relb;
  a.rowmap = p.tab->d_rowmap;
  a.out = d_out;
  a.nchan = p.nchan;
  a.cc = p.tile.chan_chunk;
  a.elmax = elmax;
  a.nst = p.tile.nbuf;
  a.one = 1u;
  a.nz = rows ? nrows : 0;
  a.withhold = p.withhold_chunk;
  for (int i = 0; i < a.nz; ++i) a.z[i] = rows[i];
  dim3 grid((unsigned)p.tab->n_dm_tiles, (unsigned)ntt,
            (unsigned)(a.nz > 0 ? a.nz : 1));
  const long long timeout =
      p.wait_limit > 0 ? p.wait_limit : kDefaultWaitCycles;
  kern<<<grid, 32 * (WT * WD + 1), smem, s>>>(a, p.d_err, timeout);
  return cudaGetLastError();
}

}  // namespace

size_t dedisp_il_smem_bytes(int chan_chunk, int dm_tile, int elmax,
                            int nst) {
  return (size_t)IlLayout(chan_chunk, dm_tile, elmax, nst).total;
}

int dedisp_il_max_stages() { return kIlMaxStages; }

IlLaunch il_launch_of(const Plan &p) {
  IlLaunch v;
  v.tile = p.tile;
  v.tab = &p.tab;
  v.nchan = p.nchan;
  v.nbits = p.nbits;
  v.d_err = p.d_err;
  v.d_il = p.d_il;
  v.wait_limit = p.wait_limit > 0 ? p.wait_limit : kDefaultWaitCycles;
  v.withhold_chunk = p.withhold_chunk;
  return v;
}

cudaError_t launch_interleave(const Plan &p, const void *d_cm, int64_t pitch,
                              int64_t nvalid, int64_t ypitch, cudaStream_t s) {
  return launch_interleave(il_launch_of(p), d_cm, pitch, nvalid, ypitch, s);
}

cudaError_t launch_interleave(const IlLaunch &p, const void *d_cm,
                              int64_t pitch, int64_t nvalid, int64_t ypitch,
                              cudaStream_t s, int64_t ring, int64_t t0,
                              void *ydst) {
  const int S = dedisp_segment(p.tile);
  const dim3 grid((unsigned)((ypitch / 4 + 255) / 256), (unsigned)p.nchan);
  uint32_t *y = static_cast<uint32_t *>(ydst ? ydst : p.d_il);
  const bool al16 = (reinterpret_cast<uintptr_t>(d_cm) & 15) == 0 &&
                    pitch % 16 == 0 && S % 16 == 0 &&
                    (ring <= 0 || (ring % 16 == 0 && t0 % 16 == 0));
  if (p.nbits == 8 && al16) {
    const dim3 g16((unsigned)(((ypitch + 15) / 16 + 255) / 256),
                   (unsigned)p.nchan);
    interleave16_u8_kernel<<<g16, 256, 0, s>>>(
        static_cast<const uint8_t *>(d_cm), pitch, nvalid, S, y, ypitch, ring,
        t0);
  } else if (p.nbits == 8)
    interleave_kernel<uint8_t><<<grid, 256, 0, s>>>(
        static_cast<const uint8_t *>(d_cm), pitch, nvalid, S, y, ypitch, ring,
        t0);
  else
    interleave_kernel<uint16_t><<<grid, 256, 0, s>>>(
        static_cast<const uint16_t *>(d_cm), pitch, nvalid, S, y, ypitch, ring,
        t0);
  return cudaGetLastError();
}

bool unpack_interleave_fused(const Plan &p) {
  return p.nbits == 8 && p.nchan % 16 == 0;
}

cudaError_t launch_unpack_interleave(const Plan &p, const void *d_in,
                                     int64_t nsamp_in, int64_t ypitch,
                                     cudaStream_t s) {
  const int S = dedisp_segment(p.tile);
  const int64_t nt = (ypitch + kIlTS - 1) / kIlTS;
  const unsigned nc = (unsigned)((p.nchan + kIlTC - 1) / kIlTC);
  // time tiles along y while they fit its 65535 limit
  const int time_on_y = nt <= 65535;
  const dim3 grid = time_on_y ? dim3(nc, (unsigned)nt) : dim3((unsigned)nt, nc);
  unpack_interleave_u8_kernel<<<grid, 256, 0, s>>>(
      static_cast<const uint8_t *>(d_in), nsamp_in, p.nchan, S,
      static_cast<uint32_t *>(p.d_il), ypitch, time_on_y);
  return cudaGetLastError();
}

cudaError_t launch_dedisperse_il(const Plan &p, int64_t ypitch,
                                 int64_t nsamp_out, int32_t *d_out,
                                 cudaStream_t s, int elmax, size_t smem) {
  return launch_dedisperse_il(il_launch_of(p), ypitch, nsamp_out, d_out, s,
                              elmax, smem);
}

cudaError_t launch_dedisperse_il(const IlLaunch &p, int64_t ypitch,
                                 int64_t nsamp_out, int32_t *d_out,
                                 cudaStream_t s) {
  int rawmax, elmax;
  dedisp_buffer_sizes(p.tile, p.tab->span_max, p.nbits, &rawmax, &elmax);
  return launch_dedisperse_il(p, ypitch, nsamp_out, d_out, s, elmax,
                              dedisp_smem_bytes(p.tile, p.tab->span_max,
                                                p.nbits));
}

namespace {
cudaError_t launch_il_dispatch(const IlLaunch &p, int64_t ypitch,
                               int64_t nsamp_out, int32_t *d_out,
                               cudaStream_t s, int elmax, size_t smem,
                               int64_t out_pitch, const IlRows *rows,
                               int nrows);
}  // namespace

cudaError_t launch_dedisperse_il_rows(const IlLaunch &p, int64_t ypitch,
                                      int64_t nsamp_out, int64_t out_pitch,
                                      const IlRows *rows, int nrows,
                                      cudaStream_t s) {
  if (!rows || nrows < 1 || nrows > kIlMaxRows) return cudaErrorInvalidValue;
  int rawmax, elmax;
  dedisp_buffer_sizes(p.tile, p.tab->span_max, p.nbits, &rawmax, &elmax);
  return launch_il_dispatch(
      p, ypitch, nsamp_out, nullptr, s, elmax,
      dedisp_smem_bytes(p.tile, p.tab->span_max, p.nbits), out_pitch, rows,
      nrows);
}

cudaError_t launch_dedisperse_il(const IlLaunch &p, int64_t ypitch,
                                 int64_t nsamp_out, int32_t *d_out,
                                 cudaStream_t s, int elmax, size_t smem) {
  return launch_il_dispatch(p, ypitch, nsamp_out, d_out, s, elmax, smem, 0,
                            nullptr, 0);
}

namespace {
cudaError_t launch_il_dispatch(const IlLaunch &p, int64_t ypitch,
                               int64_t nsamp_out, int32_t *d_out,
                               cudaStream_t s, int elmax, size_t smem,
                               int64_t out_pitch, const IlRows *rows,
                               int nrows) {
  const int wt = p.tile.wt, wd = p.tile.wd, rd = p.tile.rd;
  const int ept = dedisp_elems_per_thread(p.tile);
#define DDSP_IL(WT_, WD_, RD_, E_, T_)                                      \
  if (wt == WT_ && wd == WD_ && rd == RD_ && ept == E_)                     \
    return launch_il_t<WT_, WD_, RD_, E_, T_>(p, ypitch, nsamp_out, d_out,  \
                                              s, elmax, smem, out_pitch,    \
                                              rows, nrows);
  if (p.nbits == 8) {
    DDSP_IL(8, 2, 8, 4, uint8_t)     // wide: 16 consumer warps, E = 32 / RD
    DDSP_IL(16, 1, 8, 4, uint8_t)
    DDSP_IL(4, 4, 8, 4, uint8_t)
    DDSP_IL(4, 4, 4, 8, uint8_t)
    DDSP_IL(8, 2, 4, 8, uint8_t)
    DDSP_IL(16, 1, 4, 8, uint8_t)
    DDSP_IL(4, 2, 8, 4, uint8_t)     // 8 consumer warps, E = 4
    DDSP_IL(8, 1, 8, 4, uint8_t)
    DDSP_IL(2, 4, 8, 4, uint8_t)
    DDSP_IL(4, 2, 4, 4, uint8_t)
    DDSP_IL(8, 1, 4, 4, uint8_t)
    DDSP_IL(2, 4, 4, 4, uint8_t)
  } else {
    DDSP_IL(4, 4, 4, 8, uint16_t)
    DDSP_IL(8, 2, 4, 8, uint16_t)
    DDSP_IL(16, 1, 4, 8, uint16_t)
    DDSP_IL(4, 2, 4, 4, uint16_t)
    DDSP_IL(8, 1, 4, 4, uint16_t)
    DDSP_IL(2, 4, 4, 4, uint16_t)
  }
#undef DDSP_IL
  return cudaErrorInvalidValue;
}
}  // namespace

}  // namespace ddsp
