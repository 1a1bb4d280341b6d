// ws_item.cuh -- one work item of the warp-specialised dedispersion
// (Sec.3.2): out[k][t] = sum_c x[c][t + d[k][c]] for one DM tile x one time
// tile of one beam, exact in int32.  Used by the per-plan kernel
// (k_dedisp_ws.cu, one item per block) and by the persistent multi-beam
// kernel (k_batch.cu, items taken from a device work queue).
//
//   * producer warps (kWsProdWarps): warp w owns the chunks G with
//     G % kWsProdWarps == w; one lane per channel issues 1-D TMA bulk copies
//     of the chunk's raw windows into one of the warp's own raw stages
//     (`nbuf`, a multiple of kWsProdWarps; transaction mbarrier), then the
//     warp relayouts the chunk into element buffer G & 1 -- element i =
//     {x[i], x[i+S], x[i+2S], x[i+3S]} so a 32-bit shared load at any delay
//     yields four output times -- and copies its delay offsets beside it;
//     the producer warps never wait for each other;
//   * consumer warps (WT x WD): SWAR accumulation of two channels per step,
//     A += wa + wb (whole words, mod 2^32) and B += p(wa) + p(wb) with p(w) =
//     {b1, 0, b3, 0} (one byte permute against zero), releasing each element
//     buffer through its "empty" mbarrier.  For <= 256 channels B's 16-bit
//     halves are the exact sums of bytes 1 and 3, and A - (B << 8) holds
//     those of bytes 0 and 2 (each < 2^16), so every <= 256 channels the
//     four sums are recovered and added into the output array (uint8: the
//     first time stored, then by reductions), or kept in registers
//     (uint16).
// The mbarrier phases run on a chunk counter that continues across the
// items a block processes (`jbase`).  Each beam carries its own channel
// chunk and buffer extents, so items of different beams lay out the same
// shared memory differently; an item starts only after every role has
// finished the previous one, so no copy of one layout is in flight when the
// next begins.  Every wait is bounded; a role that gives up records a
// timeout, drains its own copies in flight (bounded) and returns false.
#pragma once

#include "dev_util.cuh"
#include "internal.h"

namespace ddsp {

constexpr int kWsProdWarps = 2;

// Shared-memory layout (bytes, 16-aligned offsets):
//   [0, 64)                      mbarriers: raw_full[4], elem_full[2],
//                                elem_empty[2]
//   [64, 80)                     scratch words (work-item broadcast)
//   raw_rel[nbuf][rel_stride]    delay offsets as copied with a raw stage
//   raw[nbuf][cc][rawmax]        raw channel windows
//   erel[2][rel_stride]          offsets beside each element buffer
//   elem[2][cc][elmax]           interleaved elements (uint32)
struct WsLayout {
  int raw_rel_off, rel_stride, raw_off, erel_off, elem_off, elem_stride, total;
  __host__ __device__ WsLayout(int cc, int dt, int rawmax, int elmax,
                               int nbuf) {
    raw_rel_off = 80;
    rel_stride = ((cc * dt * 4 + 15) / 16) * 16;
    raw_off = raw_rel_off + nbuf * rel_stride;
    erel_off = raw_off + nbuf * cc * rawmax;
    elem_off = erel_off + 2 * rel_stride;
    elem_stride = cc * elmax * 4;
    total = elem_off + 2 * elem_stride;
  }
};

// ---------------------------------------------------------------------------
// Consumer arithmetic shared by the warp-specialised kernels.  A consumer
// thread owns RD DM trials x E interleaved elements (i0 + 32 e, e < E) of
// one time tile; element i holds SPE samples, i + m S for m < SPE.  Each DM
// offset serves E loads, so a larger E spends fewer offset loads and
// address adds per operand.

// A 1 the compiler cannot see (a device variable the host could change):
// x * ws_one() + y is an integer multiply-add, which runs on the FMA pipe,
// while x + y would take the integer ALU pipe the byte permutes also use.
static __device__ uint32_t g_ws_one = 1u;
__device__ __forceinline__ uint32_t ws_one() { return g_ws_one; }

// SWAR partials (uint8: A, B, flushed every <= 256 channels) or int32
// totals (uint16: two 16-bit samples per element, exact in int32); E
// elements per thread.
template <int RD, int SPE, int E = kElemPerThread>
struct WsAcc {
  uint32_t A[RD][E], B[RD][E];
  int32_t tot[SPE != 4 ? RD : 1][E][SPE];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int r = 0; r < RD; ++r)
#pragma unroll
      for (int e = 0; e < E; ++e) {
        A[r][e] = 0;
        B[r][e] = 0;
        if constexpr (SPE != 4) {
#pragma unroll
          for (int m = 0; m < SPE; ++m) tot[r][e][m] = 0;
        }
      }
  }
};

// Accumulate `ncur` staged channels: channel q's elements start at
// ebase + q * elmax * 4 (ebase already points at this thread's element
// i0), its DM trial r's byte offset is rel[q * dt + r] (rel already points
// at this warp's first trial; 16-byte aligned).  Two channels per step
// (3-input adds), then a lone last channel.
//
// uint8 per pair of words: A += wa + wb (one 3-input add on the ALU pipe),
// B += p(wa) + p(wb) as two multiply-adds by `one` (== 1, from ws_one())
// on the FMA pipe, and the two byte permutes on the ALU pipe: 3 ALU and 2
// FMA operations per 8 sample adds, where all-ALU would be 4 against the
// half-rate ALU pipe's 64 operations per SM clock.
// (i0: this thread's first element, for the bounds-checked build: every
// element it reads of a channel, i0 + rel/4 + 32 e for e < E, must lie in
// the channel's elmax elements; an offset that does not is replaced by one
// that reads element i0 and the violation is recorded.)
template <int RD, int SPE, int E>
__device__ __forceinline__ void ws_accumulate(WsAcc<RD, SPE, E> &acc,
                                              const int32_t *rel, int dt,
                                              const unsigned char *ebase,
                                              int elmax, int ncur,
                                              uint32_t one, int i0 = 0) {
  auto offsets = [&](int q, int(&rr)[RD]) {
#pragma unroll
    for (int h = 0; h < RD; h += 4) {
      const int4 ro = *reinterpret_cast<const int4 *>(rel + q * dt + h);
      rr[h] = ro.x;
      rr[h + 1] = ro.y;
      rr[h + 2] = ro.z;
      rr[h + 3] = ro.w;
    }
#ifdef DDSP_BOUNDS_CHECK
#pragma unroll
    for (int h = 0; h < RD; ++h) {
      const int64_t last = (int64_t)i0 + rr[h] / 4 + 32 * (E - 1);
      if (!DDSP_BC(rr[h] >= 0 && (rr[h] & 3) == 0 && last < elmax, kBcIlElem,
                   last))
        rr[h] = 0;
    }
#endif
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
          acc.A[r][e] += wa + wb;
          acc.B[r][e] = __byte_perm(wa, 0u, 0x4341) * one + acc.B[r][e];
          acc.B[r][e] = __byte_perm(wb, 0u, 0x4341) * one + acc.B[r][e];
        } else {
          acc.tot[r][e][0] += (int32_t)((wa & 0xFFFFu) + (wb & 0xFFFFu));
          acc.tot[r][e][1] += (int32_t)((wa >> 16) + (wb >> 16));
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
          acc.A[r][e] += wa;
          acc.B[r][e] += __byte_perm(wa, 0u, 0x4341);
        } else {
          acc.tot[r][e][0] += (int32_t)(wa & 0xFFFFu);
          acc.tot[r][e][1] += (int32_t)(wa >> 16);
        }
      }
    }
  }
}

// uint8: unpack the SWAR partials (<= 256 channels since the last flush)
// into the output rows rowmap[r] (-1: padding trial) at times t0 + 32 e +
// m S; the item's first flush stores, later ones are fire-and-forget
// reductions (integer adds in any order give the same total).
template <int RD, int E>
__device__ __forceinline__ void ws_flush(WsAcc<RD, 4, E> &acc,
                                         const int32_t *rowmap, int32_t *out,
                                         int64_t out_pitch, int64_t t0, int S,
                                         int64_t nsamp_out, bool first) {
#pragma unroll
  for (int r = 0; r < RD; ++r) {
    const int row = __ldg(rowmap + r);
    int32_t *o = out + (int64_t)(row < 0 ? 0 : row) * out_pitch;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const uint32_t Bv = acc.B[r][e];
      const uint32_t Ev = acc.A[r][e] - (Bv << 8);  // b0 + 2^16 b2 sums
      const int32_t part[4] = {(int32_t)(Ev & 0xFFFFu), (int32_t)(Bv & 0xFFFFu),
                               (int32_t)(Ev >> 16), (int32_t)(Bv >> 16)};
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int64_t t = t0 + 32 * e + (int64_t)m * S;
        if (row >= 0 && t < nsamp_out && DDSP_BC(t >= 0, kBcIlOut, t)) {
          if (first) o[t] = part[m];
          else atomicAdd(o + t, part[m]);
        }
      }
      acc.A[r][e] = 0;
      acc.B[r][e] = 0;
    }
  }
}

// uint16: store the register totals once, after the last channel.
template <int RD, int SPE, int E>
__device__ __forceinline__ void ws_store_totals(const WsAcc<RD, SPE, E> &acc,
                                                const int32_t *rowmap,
                                                int32_t *out, int64_t out_pitch,
                                                int64_t t0, int S,
                                                int64_t nsamp_out) {
#pragma unroll
  for (int r = 0; r < RD; ++r) {
    const int row = rowmap[r];
    if (row < 0) continue;
    int32_t *o = out + (int64_t)row * out_pitch;
#pragma unroll
    for (int e = 0; e < E; ++e)
#pragma unroll
      for (int m = 0; m < SPE; ++m) {
        const int64_t t = t0 + 32 * e + (int64_t)m * S;
        if (t < nsamp_out) o[t] = acc.tot[r][e][m];
      }
  }
}

// One beam as the dedispersion sees it (device copy for the batch).  Input
// sample t + d of channel c sits at row offset t + d (ring == 0), or at
// (t0 + t + d) mod ring for a ring buffer whose rows carry, past `ring`, a
// copy of their first bytes so no staged window wraps.
struct WsBeam {
  const void *cm;           // channel-major rows [nchan][pitch]
  int64_t pitch;
  int64_t nsamp_out;
  int64_t ring;             // ring length in samples, 0 = linear rows
  int64_t t0;               // ring position of output sample 0's input
  int64_t out_pitch;        // output row pitch (samples)
  const int2 *desc;         // [n_dm_tiles][nchan] {window start, bytes}
  const int32_t *relb;      // [n_dm_tiles][nchan][DT] element-byte offsets
  const int32_t *rowmap;    // [n_dm_tiles*DT] output row or -1
  int32_t *out;             // [ndm][out_pitch]
  int nchan;
  int n_dm_tiles;
  int n_time_tiles;
  int cc;                   // channels per chunk (<= 32)
  int rawmax;               // bytes of one raw channel window
  int elmax;                // elements of one relayouted channel
  int pad[2];
};

__device__ __forceinline__ void ws_init_barriers(unsigned char *smem,
                                                 int nbuf, int nc) {
  uint64_t *raw_full = reinterpret_cast<uint64_t *>(smem);
  uint64_t *elem_full = raw_full + 4;
  uint64_t *elem_empty = raw_full + 6;
  for (int b = 0; b < nbuf; ++b) mbar_init(&raw_full[b], 1);
  for (int b = 0; b < 2; ++b) {
    mbar_init(&elem_full[b], 1);   // the one producer warp of the chunk
    mbar_init(&elem_empty[b], nc);
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Process DM tile g x time tile starting at output sample T0 of beam `a`.
// `jbase` is the number of chunks this block processed before (same value
// in every thread).  Returns false if this thread's role gave up.
template <int WT, int WD, int RD, typename T>
__device__ __forceinline__ bool ws_item(const WsBeam &a, int g, int64_t T0,
                                        int jbase, unsigned char *smem,
                                        int nbuf, int32_t *err,
                                        long long timeout_cycles) {
  constexpr int SPE = 4 / sizeof(T);   // samples per element
  constexpr int E = kElemPerThread;
  constexpr int S = 32 * E * WT;       // elements per segment
  constexpr int DT = RD * WD;          // DM trials per tile
  constexpr int NC = WT * WD;          // consumer warps
  constexpr int NP = kWsProdWarps;
  const int cc = a.cc, rawmax = a.rawmax, elmax = a.elmax;
  const WsLayout L(cc, DT, rawmax, elmax, nbuf);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint64_t *raw_full = reinterpret_cast<uint64_t *>(smem);
  uint64_t *elem_full = raw_full + 4;
  uint64_t *elem_empty = raw_full + 6;
  unsigned char *raw_rel = smem + L.raw_rel_off;
  unsigned char *raw = smem + L.raw_off;
  int32_t *erel = reinterpret_cast<int32_t *>(smem + L.erel_off);
  unsigned char *elem = smem + L.elem_off;
  const int rel_words = L.rel_stride / 4;

  const T *cm = static_cast<const T *>(a.cm);
  const int nchan = a.nchan;
  const int64_t nsamp_out = a.nsamp_out;
  const int nchunks = (nchan + cc - 1) / cc;
  const int2 *desc_g = a.desc + (int64_t)g * nchan;
  const int32_t *rel_g = a.relb + (int64_t)g * nchan * DT;

  if (warp >= NC) {
    // ============================ producers ============================
    // Producer warp pw owns the chunks G = jbase + j with G % NP == pw: it
    // waits for their windows, relayouts all their channels into element
    // buffer G & 1 and issues their refills, so the producer warps never
    // wait for each other.  nbuf is a multiple of NP: a warp's raw stages
    // are its own.
    const int pw = warp - NC;
    int2 nd = make_int2(0, 0);  // next copy descriptor of this lane's channel
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
      const int st = (jbase + j) % nbuf;
      if (lane == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&raw_full[st], total);
      }
      __syncwarp();
      if (v) {
        int64_t pos = T0 + nd.x;
        if (a.ring > 0) pos = (a.t0 + pos) % a.ring;
        bulk_g2s(raw + (st * cc + lane) * rawmax,
                 cm + (int64_t)(c0 + lane) * a.pitch + pos, nb, &raw_full[st]);
      }
      if (lane == 0)
        bulk_g2s(raw_rel + st * L.rel_stride, rel_g + (int64_t)c0 * DT,
                 relbytes, &raw_full[st]);
    };
    const int j0 = ((pw - jbase) % NP + NP) % NP;   // first own chunk
    int last_issued = -1;
    int jn = j0;
    for (; jn < nbuf; jn += NP) {
      if (jn < nchunks) {
        load_desc(jn);
        issue(jn);
        last_issued = jn;
      }
    }
    load_desc(jn);
    int j = j0;
    bool failed = false;
    for (; j < nchunks; j += NP) {
      const int G = jbase + j;
      const int st = G % nbuf, b = G & 1;
      const int ncur = min(cc, nchan - j * cc);
      bool ok = mbar_wait(&raw_full[st], (uint32_t)((G / nbuf) & 1),
                          timeout_cycles);
      ok = ok && mbar_wait(&elem_empty[b], (uint32_t)(((G >> 1) & 1) ^ 1),
                           timeout_cycles);
      if (!ok) {
        failed = true;
        break;
      }
      const int32_t *rs =
          reinterpret_cast<const int32_t *>(raw_rel + st * L.rel_stride);
      int32_t *er = erel + b * rel_words;
      for (int i = lane; i < ncur * DT; i += 32) er[i] = rs[i];
      const unsigned char *rb = raw + st * cc * rawmax;
      uint32_t *eb = reinterpret_cast<uint32_t *>(elem + b * L.elem_stride);
      for (int q = 0; q < ncur; ++q) {
        const unsigned char *rq = rb + q * rawmax;
        uint32_t *eq = eb + q * elmax;
        const int span = rs[q * DT + DT - 1] >> 2;
        if constexpr (SPE == 4) {
          // groups of 4 elements: lane l takes groups l + 64m and
          // l + 64m + 32 per step, all 8 loads issued before the stores so
          // their latencies overlap; a lone last group is done after the
          // loop.  Loads and stores use fixed offsets from two running
          // pointers.
          const int nq = (S + span + 3) >> 2;
          constexpr int SW = S / 4;   // words per segment
          const uint32_t *rw = reinterpret_cast<const uint32_t *>(rq) + lane;
          uint4 *ev = reinterpret_cast<uint4 *>(eq) + lane;
          int i4 = lane;
          for (; i4 + 32 < nq; i4 += 64, rw += 64, ev += 64) {
            const uint32_t a0 = rw[0], a1 = rw[SW], a2 = rw[2 * SW],
                           a3 = rw[3 * SW];
            const uint32_t b0 = rw[32], b1 = rw[32 + SW], b2 = rw[32 + 2 * SW],
                           b3 = rw[32 + 3 * SW];
            ev[0] = transpose4x4(a0, a1, a2, a3);
            ev[32] = transpose4x4(b0, b1, b2, b3);
          }
          if (i4 < nq) ev[0] = transpose4x4(rw[0], rw[SW], rw[2 * SW], rw[3 * SW]);
        } else {
          const int nq = (S + span + 1) >> 1;
          for (int i2 = lane; i2 < nq; i2 += 32) {
            const unsigned char *p = rq + 4 * i2;
            const uint32_t w0 = *reinterpret_cast<const uint32_t *>(p);
            const uint32_t w1 = *reinterpret_cast<const uint32_t *>(p + 2 * S);
            uint2 o;
            o.x = __byte_perm(w0, w1, 0x5410);
            o.y = __byte_perm(w0, w1, 0x7632);
            *reinterpret_cast<uint2 *>(eq + 2 * i2) = o;
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&elem_full[b]);
      if (j + nbuf < nchunks) {
        issue(j + nbuf);
        last_issued = j + nbuf;
        load_desc(j + nbuf + NP);
      }
    }
    if (failed && lane == 0) {
      atomicExch(err, kErrTimeout);
      for (int jj = j; jj <= last_issued; jj += NP) {
        const int G = jbase + jj;
        mbar_wait(&raw_full[G % nbuf], (uint32_t)((G / nbuf) & 1),
                  timeout_cycles);
      }
    }
    return !failed;
  }

  // ============================= consumers =============================
  const int wt = warp % WT, wd = warp / WT;
  const int i0 = 32 * E * wt + lane;  // first element of this thread
  const uint32_t one = ws_one();
  WsAcc<RD, SPE> acc;
  acc.zero();
  bool first_flush = true;
  int since = 0;

  for (int j = 0; j < nchunks; ++j) {
    const int G = jbase + j;
    const int b = G & 1;
    const int ncur = min(cc, nchan - j * cc);
    if (!mbar_wait(&elem_full[b], (uint32_t)((G >> 1) & 1), timeout_cycles)) {
      if (lane == 0) atomicExch(err, kErrTimeout);
      return false;
    }
    ws_accumulate(acc, erel + b * rel_words + RD * wd, DT,
                  elem + b * L.elem_stride + 4 * i0, elmax, ncur, one, i0);
    __syncwarp();
    if (lane == 0) mbar_arrive(&elem_empty[b]);
    if constexpr (SPE == 4) {
      since += ncur;
      if (since + cc > 256 || j == nchunks - 1) {
        ws_flush(acc, a.rowmap + g * DT + RD * wd, a.out, a.out_pitch,
                 T0 + i0, S, nsamp_out, first_flush);
        first_flush = false;
        since = 0;
      }
    }
  }
  if constexpr (SPE != 4)
    ws_store_totals(acc, a.rowmap + g * DT + RD * wd, a.out, a.out_pitch,
                    T0 + i0, S, nsamp_out);
  return true;
}

}  // namespace ddsp
