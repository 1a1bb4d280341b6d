// server.cu -- streaming search of many beams of one shape (the real-time
// ring-buffer design of Sec.2.1 and Ch.3: each beam delivers a block of B new
// spectra at a time and every block is dedispersed and searched as soon as
// the GPU is free, alongside whatever other beams have a block waiting).
//
// Per beam the server holds
//   * a channel-major ring of `slots` blocks (slots = ceil(D16 / B) + 1, D16 =
//     the largest delay rounded up to 16 samples: the B + D16 input samples a
//     block's step reads plus the rest of one block) whose rows carry past the
//     ring a copy of their first M bytes, M >= the longest window one
//     dedispersion work item stages, so a staged window never wraps;
//   * the carry [ndm][C]: the last C output samples of the previous block
//     (C = the widest boxcar minus one, rounded up to 4), so every boxcar that
//     starts in the new block is complete;
//   * per-window statistics and two candidate buffers (by block parity), so a
//     block's candidates can be read while the next block is processed.
// The series [ndm][C + B] a block is searched on lives only during its step,
// in one of G series slots the server shares among the beams (G = the
// group size: a step runs its beam-blocks in groups of G, each group's
// carry in, dedispersion, search and carry out one after the other), so a
// beam costs its ring and a few MB, not a series of its own.
// Block j's input lands in slot j % slots.  Its step dedisperses output
// samples [s_j, s_j + B) with s_j = j*B - D16 (input [s_j, s_j + B + D) is
// then resident: blocks j-slots+1 .. j), writing series columns [C, C + B),
// and searches start times [0, B) of the whole series (global time
// s_j - C + t).  Samples before the stream's start read as zero.  Pushing
// block j overwrites the slot of block j - slots, which the step of block
// j - 1 is the last to read, so a push waits for that step.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "host.h"
#include "ws_item.cuh"

using namespace ddsp;

namespace {

constexpr int kStepEvents = 64;

// Series slots of the relayout mode's groups (one persistent launch each).
constexpr int kRelayoutGroup = 16;

struct ServerBeam {
  bool live = false;
  uint8_t *ring = nullptr;      // [nchan][pitch]
  int32_t *carry = nullptr;     // [ndm][C]
  int series_slot = -1;         // series slot of the last step (G slots)
  int64_t *m2 = nullptr, *mad4 = nullptr;
  ddsp_cand *cands = nullptr;   // [2][cap]
  int64_t pushed = 0;           // blocks ingested
  int64_t processed = 0;        // blocks taken by enqueued steps
  int64_t step_of[4] = {-1, -1, -1, -1};  // step of block j, by j % 4
  int64_t push_seq[2] = {0, 0};  // server-wide push order of block j, by j % 2
  cudaEvent_t ev_push[2] = {nullptr, nullptr};  // by block parity
};

}  // namespace

struct ddsp_server {
  int device = 0;
  ddsp_plan *plan = nullptr;
  int64_t B = 0, C = 0, D16 = 0, R = 0, M = 0, pitch = 0, ncols = 0, nwin = 0;
  int slots = 0;
  DedispTile tile;
  DedispTables tab;
  int cc = 0, rawmax = 0, elmax = 0, grid = 0, ipb = 0, ntt = 0;
  size_t smem = 0, sps_smem = 0;
  int64_t sps_cap = 0;
  int max_beams = 0;
  int64_t reserve = 0;
  uint32_t cap = 0;
  std::vector<ServerBeam> beams;
  uint32_t *d_counts = nullptr;  // [max_beams][2]
  int32_t *d_err = nullptr;
  int *d_queue = nullptr;
  WsBeam *d_wsb[2] = {nullptr, nullptr};
  SpsBeam *d_sb[2] = {nullptr, nullptr};
  int32_t **d_carry[2] = {nullptr, nullptr};
  WsBeam *h_wsb[2] = {nullptr, nullptr};   // pinned staging of a step's
  SpsBeam *h_sb[2] = {nullptr, nullptr};   // descriptors, by step parity
  int32_t **h_carry[2] = {nullptr, nullptr};
  // series slots [G][ndm][ncols] shared by the beam-blocks of a group
  int G = 0;
  int32_t *d_pool = nullptr;
  cudaEvent_t ev_step[kStepEvents] = {};
  int64_t nsteps = 0;
  int64_t npushes = 0;
  // interleaved mode: waiting beam-blocks are interleaved from their rings
  // into `il_slots` staging slots and dedispersed by one interleaved launch
  // per group of slots
  int mode = DDSP_SERVER_RELAYOUT;
  DedispTile il_tile;
  DedispTables il_tab;
  int il_slots = 0;
  int64_t ypitch = 0;
  size_t slot_bytes = 0;
  uint8_t *d_il = nullptr;
};

namespace {

int64_t floor_mod(int64_t a, int64_t m) {
  const int64_t r = a % m;
  return r < 0 ? r + m : r;
}

int64_t beam_bytes(const ddsp_server &S) {
  const Plan &p = S.plan->p;
  return (int64_t)p.nchan * S.pitch + (int64_t)p.ndm * S.C * 4 +
         2 * (int64_t)p.ndm * S.nwin * 8 + 2 * (int64_t)S.cap * 16;
}

void free_beam(ServerBeam &b) {
  cudaFree(b.ring);
  cudaFree(b.carry);
  cudaFree(b.m2);
  cudaFree(b.mad4);
  cudaFree(b.cands);
  for (auto &e : b.ev_push)
    if (e) cudaEventDestroy(e);
  b = ServerBeam{};
}

void server_release(ddsp_server &S) {
  for (auto &b : S.beams)
    if (b.live) free_beam(b);
  free_tables(S.tab);
  free_tables(S.il_tab);
  cudaFree(S.d_il);
  cudaFree(S.d_pool);
  cudaFree(S.d_counts);
  cudaFree(S.d_err);
  cudaFree(S.d_queue);
  for (int i = 0; i < 2; ++i) {
    cudaFree(S.d_wsb[i]);
    cudaFree(S.d_sb[i]);
    cudaFree(S.d_carry[i]);
    cudaFreeHost(S.h_wsb[i]);
    cudaFreeHost(S.h_sb[i]);
    cudaFreeHost(S.h_carry[i]);
  }
  for (auto &e : S.ev_step)
    if (e) cudaEventDestroy(e);
}

// Event of step `id` (a later step's record of the same event only makes a
// wait on it longer, never wrong: steps complete in order).
cudaEvent_t step_event(const ddsp_server &S, int64_t id) {
  return S.ev_step[id % kStepEvents];
}

// (Re)allocate the G series slots; nothing may be running on them.
int set_pool(ddsp_server &S, int G) {
  const Plan &p = S.plan->p;
  cudaDeviceSynchronize();
  cudaFree(S.d_pool);
  S.d_pool = nullptr;
  S.G = 0;
  cudaError_t e = cudaMalloc(&S.d_pool, (size_t)G * p.ndm * S.ncols * 4);
  if (e != cudaSuccess) return cuda_rc(e);
  S.G = G;
  for (auto &b : S.beams) b.series_slot = -1;
  return DDSP_OK;
}

int32_t *pool_slot(const ddsp_server &S, int q) {
  const Plan &p = S.plan->p;
  return S.d_pool + (size_t)q * p.ndm * S.ncols;
}

// Candidates tiles tried in order when the caller leaves the choice to the
// server: the first whose windows fit two blocks per SM for this shape.
const DedispTile kServerTiles[] = {
    {4, 2, 8, 8, 2, kTileWarpSpecialized}, {8, 1, 8, 4, 2, kTileWarpSpecialized},
    {4, 2, 8, 4, 2, kTileWarpSpecialized}, {8, 1, 4, 4, 2, kTileWarpSpecialized},
    {4, 2, 4, 4, 2, kTileWarpSpecialized}, {8, 1, 4, 2, 2, kTileWarpSpecialized},
    {8, 1, 4, 1, 2, kTileWarpSpecialized}};

// Fit tile t to the server's shape: per-beam chunk (largest <= t.chan_chunk
// within the two-block budget, else one block), buffers, grid.
int server_apply_tile(ddsp_server &S, const DedispTile &t) {
  const Plan &p = S.plan->p;
  if (!dedisp_tile_supported(t, 8) || !(t.flags & kTileWarpSpecialized))
    return DDSP_E_INVALID_ARG;
  const int TT = dedisp_time_tile(t, 8);
  if (S.B % TT) return DDSP_E_INVALID_ARG;
  const int span = span_for(p, t.dm_tile());
  int rawmax, elmax;
  dedisp_buffer_sizes(t, span, 8, &rawmax, &elmax);
  int cc = 0;
  size_t smem = 0;
  for (size_t budget : {kSmemBudgetTwoBlocks, kSmemBudgetOneBlock}) {
    for (int c = t.chan_chunk; c >= 1 && !cc; --c) {
      const size_t sm =
          dedisp_ws_smem_bytes(c, t.dm_tile(), rawmax, elmax, t.nbuf);
      if (sm <= budget) {
        cc = c;
        smem = sm;
      }
    }
    if (cc) break;
  }
  if (!cc) return DDSP_E_INVALID_ARG;
  int rc = build_tables_for(p, t, S.tab);
  if (rc != DDSP_OK) return rc;
  int per_sm = persistent_blocks_per_sm(t, smem);
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, S.device);
  if (per_sm <= 0 || nsm <= 0) return DDSP_E_INVALID_ARG;
  S.tile = t;
  S.cc = cc;
  S.rawmax = rawmax;
  S.elmax = elmax;
  S.smem = smem;
  S.grid = per_sm * nsm;
  S.ntt = (int)(S.B / TT);
  S.ipb = S.tab.n_dm_tiles * S.ntt;
  // the longest staged window, rounded up: the mirrored row tail
  S.M = round_up(dedisp_copy_bytes(t, S.tab.span_max, 8) + 16, 128);
  return DDSP_OK;
}

// The interleaved tile of the interleaved mode: its time tile divides the
// block.
DedispTile server_il_tile(const ddsp_server &S) {
  const Plan &p = S.plan->p;
  return fit_interleaved_tile([&](int tt) { return S.B % tt == 0; },
                              [&](int dt) { return span_for(p, dt); });
}

// The interleaved mode's dedispersion of one group of n <= il_slots waiting
// beam-blocks: each block's window of its ring (logical samples [0, B + D16)
// from ring position t0) is interleaved into a staging slot, then one launch
// covers the group (blockIdx.z = slot) and writes series slot q's columns
// [C, C + B).  Stream order keeps a slot's next interleave behind the launch
// that read it.
cudaError_t server_dedisperse_il(ddsp_server &S, const int *beams,
                                 const int64_t *t0, int n, cudaStream_t s) {
  const Plan &p = S.plan->p;
  IlLaunch v;
  v.tile = S.il_tile;
  v.tab = &S.il_tab;
  v.nchan = p.nchan;
  v.nbits = 8;
  v.d_err = S.d_err;
  cudaError_t e = cudaSuccess;
  IlRows rows[kIlMaxRows];
  for (int q = 0; q < n && e == cudaSuccess; ++q) {
    const ServerBeam &b = S.beams[beams[q]];
    uint8_t *slot = S.d_il + (size_t)q * S.slot_bytes;
    e = launch_interleave(v, b.ring, S.pitch, S.B + S.D16, S.ypitch, s, S.R,
                          t0[q], slot);
    rows[q].y = reinterpret_cast<const uint32_t *>(slot);
    rows[q].out = pool_slot(S, q) + S.C;
  }
  if (e == cudaSuccess)
    e = launch_dedisperse_il_rows(v, S.ypitch, S.B, S.ncols, rows, n, s);
  return e;
}

}  // namespace

extern "C" {

int ddsp_server_set_mode(ddsp_server *S, int mode, int staging_slots) {
  if (!S || (mode != DDSP_SERVER_RELAYOUT && mode != DDSP_SERVER_INTERLEAVED))
    return DDSP_E_INVALID_ARG;
  if (mode == DDSP_SERVER_INTERLEAVED &&
      (staging_slots < 1 || staging_slots > kIlMaxRows))
    return DDSP_E_INVALID_ARG;
  DeviceGuard g(S->device);
  cudaDeviceSynchronize();   // no step may still read the staging slots
  if (mode == DDSP_SERVER_RELAYOUT) {
    const int rc = set_pool(*S, kRelayoutGroup);
    if (rc != DDSP_OK) return rc;
    free_tables(S->il_tab);
    cudaFree(S->d_il);
    S->d_il = nullptr;
    S->il_slots = 0;
    S->mode = mode;
    return DDSP_OK;
  }
  const DedispTile t = server_il_tile(*S);
  if (t.wt == 0) return DDSP_E_INVALID_ARG;
  const Plan &p = S->plan->p;
  const int64_t ypitch = round_up(S->B + S->D16 + 64, 128);
  const size_t slot_bytes = (size_t)p.nchan * ypitch * 4;
  DedispTables tab;
  int rc = build_tables_for(p, t, tab);
  if (rc != DDSP_OK) return rc;
  uint8_t *d_il = nullptr;
  cudaError_t e = cudaMalloc(&d_il, slot_bytes * staging_slots);
  if (e != cudaSuccess) {
    free_tables(tab);
    return cuda_rc(e);
  }
  rc = set_pool(*S, staging_slots);
  if (rc != DDSP_OK) {
    free_tables(tab);
    cudaFree(d_il);
    return rc;
  }
  free_tables(S->il_tab);
  cudaFree(S->d_il);
  S->il_tab = tab;
  S->il_tile = t;
  S->d_il = d_il;
  S->ypitch = ypitch;
  S->slot_bytes = slot_bytes;
  S->il_slots = staging_slots;
  S->mode = mode;
  return DDSP_OK;
}

int ddsp_server_get_mode(const ddsp_server *S, int *mode, int *staging_slots) {
  if (!S) return DDSP_E_INVALID_ARG;
  if (mode) *mode = S->mode;
  if (staging_slots) *staging_slots = S->il_slots;
  return DDSP_OK;
}

int ddsp_server_create(ddsp_server **out, ddsp_plan *plan,
                       int64_t block_samples, int max_beams,
                       int64_t hbm_reserve_bytes, int dm_tile,
                       int dm_per_thread, int chan_chunk, int stages) {
  if (!out || !plan || max_beams <= 0 || hbm_reserve_bytes < 0)
    return DDSP_E_INVALID_ARG;
  *out = nullptr;
  const Plan &p = plan->p;
  if (p.nbits != 8 || p.nchan % 16 != 0) return DDSP_E_INVALID_ARG;
  if (block_samples <= 0 || block_samples % 16) return DDSP_E_SHAPE;
  ddsp_server *S = new (std::nothrow) ddsp_server;
  if (!S) return DDSP_E_NOMEM;
  S->device = p.device;
  DeviceGuard g(S->device);
  S->plan = plan;
  S->B = block_samples;
  S->C = round_up(p.widths.back() - 1, 4);
  S->D16 = round_up(p.max_delay, 16);
  S->slots = (int)((S->D16 + S->B - 1) / S->B) + 1;
  S->R = S->slots * S->B;
  S->ncols = S->C + S->B;
  S->max_beams = max_beams;
  S->reserve = hbm_reserve_bytes;
  S->cap = (uint32_t)std::min<size_t>(p.cand_capacity, 0xffffffffu);
  int rc = DDSP_OK;
  if (S->B < S->C) rc = DDSP_E_SHAPE;
  if (rc == DDSP_OK) rc = search_windows(p, S->ncols, &S->nwin);
  if (rc == DDSP_OK) {
    if (dm_tile > 0) {
      DedispTile t;
      if (dm_per_thread <= 0 || dm_tile % dm_per_thread) {
        rc = DDSP_E_INVALID_ARG;
      } else {
        t.rd = dm_per_thread;
        t.wd = dm_tile / dm_per_thread;
        t.wt = t.wd > 0 ? (kThreads / 32) / t.wd : 0;
        t.chan_chunk = chan_chunk;
        t.nbuf = stages;
        t.flags = kTileWarpSpecialized;
        rc = server_apply_tile(*S, t);
      }
    } else {
      rc = DDSP_E_INVALID_ARG;
      for (const DedispTile &t : kServerTiles) {
        rc = server_apply_tile(*S, t);
        if (rc == DDSP_OK) break;
      }
    }
  }
  if (rc == DDSP_OK && S->M > S->B) rc = DDSP_E_SHAPE;  // mirror from one block
  if (rc == DDSP_OK) {
    S->pitch = round_up(S->R + S->M, 128);
    const int64_t maxlen = (p.norm_window <= 0 || S->nwin == 1)
                               ? S->ncols
                               : std::max<int64_t>(p.norm_window,
                                                   S->ncols - (S->nwin - 1) * p.norm_window);
    S->sps_smem = sps_smem_bytes(maxlen, p.widths.back());
    S->sps_cap = sps_bufcap(maxlen, p.widths.back());
    S->beams.resize(max_beams);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
      if ((e = cudaMalloc(&S->d_wsb[i], max_beams * sizeof(WsBeam))) == cudaSuccess &&
          (e = cudaMalloc(&S->d_sb[i], max_beams * sizeof(SpsBeam))) == cudaSuccess &&
          (e = cudaMalloc(&S->d_carry[i], max_beams * sizeof(int32_t *))) == cudaSuccess &&
          (e = cudaMallocHost(&S->h_wsb[i], max_beams * sizeof(WsBeam))) == cudaSuccess &&
          (e = cudaMallocHost(&S->h_carry[i], max_beams * sizeof(int32_t *))) == cudaSuccess)
        e = cudaMallocHost(&S->h_sb[i], max_beams * sizeof(SpsBeam));
    }
    if (e == cudaSuccess &&
        (e = cudaMalloc(&S->d_counts, 2 * max_beams * sizeof(uint32_t))) == cudaSuccess &&
        (e = cudaMalloc(&S->d_err, sizeof(int32_t))) == cudaSuccess)
      e = cudaMalloc(&S->d_queue, sizeof(int));
    for (int i = 0; i < kStepEvents && e == cudaSuccess; ++i)
      e = cudaEventCreateWithFlags(&S->ev_step[i], cudaEventDisableTiming);
    if (e == cudaSuccess) {
      cudaMemset(S->d_counts, 0, 2 * max_beams * sizeof(uint32_t));
      e = cudaMemset(S->d_err, 0, sizeof(int32_t));
    }
    if (e != cudaSuccess) rc = cuda_rc(e);
    if (rc == DDSP_OK) rc = set_pool(*S, kRelayoutGroup);
  }
  if (rc != DDSP_OK) {
    server_release(*S);
    delete S;
    return rc;
  }
  *out = S;
  return DDSP_OK;
}

void ddsp_server_destroy(ddsp_server *S) {
  if (!S) return;
  DeviceGuard g(S->device);
  cudaDeviceSynchronize();
  server_release(*S);
  delete S;
}

int ddsp_server_info(const ddsp_server *S, int64_t *beam_bytes_out,
                     int64_t *ring_samples, int64_t *series_cols,
                     int64_t *carry, int64_t *first_delay) {
  if (!S) return DDSP_E_INVALID_ARG;
  if (beam_bytes_out) *beam_bytes_out = beam_bytes(*S);
  if (ring_samples) *ring_samples = S->R;
  if (series_cols) *series_cols = S->ncols;
  if (carry) *carry = S->C;
  if (first_delay) *first_delay = S->D16;
  return DDSP_OK;
}

int ddsp_server_get_tile(const ddsp_server *S, int *dm_tile, int *dm_per_thread,
                         int *time_tile, int *chan_chunk, int *stages,
                         int *grid) {
  if (!S) return DDSP_E_INVALID_ARG;
  if (dm_tile) *dm_tile = S->tile.dm_tile();
  if (dm_per_thread) *dm_per_thread = S->tile.rd;
  if (time_tile) *time_tile = dedisp_time_tile(S->tile, 8);
  if (chan_chunk) *chan_chunk = S->cc;
  if (stages) *stages = S->tile.nbuf;
  if (grid) *grid = S->grid;
  return DDSP_OK;
}

int ddsp_server_admit(ddsp_server *S, int *beam) {
  if (!S || !beam) return DDSP_E_INVALID_ARG;
  *beam = -1;
  DeviceGuard g(S->device);
  int slot = -1;
  for (int i = 0; i < S->max_beams && slot < 0; ++i)
    if (!S->beams[i].live) slot = i;
  if (slot < 0) return DDSP_E_RANGE;
  size_t free_b = 0, total_b = 0;
  cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
  if (e != cudaSuccess) return cuda_rc(e);
  if ((int64_t)free_b < beam_bytes(*S) + S->reserve) return DDSP_E_NOMEM;
  const Plan &p = S->plan->p;
  ServerBeam b;
  if ((e = cudaMalloc(&b.ring, (size_t)p.nchan * S->pitch)) == cudaSuccess &&
      (e = cudaMalloc(&b.carry, (size_t)p.ndm * S->C * 4)) == cudaSuccess &&
      (e = cudaMalloc(&b.m2, (size_t)p.ndm * S->nwin * 8)) == cudaSuccess &&
      (e = cudaMalloc(&b.mad4, (size_t)p.ndm * S->nwin * 8)) == cudaSuccess &&
      (e = cudaMalloc(&b.cands, 2 * (size_t)S->cap * sizeof(ddsp_cand))) == cudaSuccess &&
      (e = cudaEventCreateWithFlags(&b.ev_push[0], cudaEventDisableTiming)) == cudaSuccess &&
      (e = cudaEventCreateWithFlags(&b.ev_push[1], cudaEventDisableTiming)) == cudaSuccess &&
      (e = cudaMemset(b.ring, 0, (size_t)p.nchan * S->pitch)) == cudaSuccess)
    e = cudaMemset(b.carry, 0, (size_t)p.ndm * S->C * 4);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_beam(b);
    return cuda_rc(e);
  }
  b.live = true;
  S->beams[slot] = b;
  *beam = slot;
  return DDSP_OK;
}

int ddsp_server_evict(ddsp_server *S, int beam) {
  if (!S || beam < 0 || beam >= S->max_beams || !S->beams[beam].live)
    return DDSP_E_INVALID_ARG;
  DeviceGuard g(S->device);
  cudaDeviceSynchronize();
  free_beam(S->beams[beam]);
  return DDSP_OK;
}

int ddsp_server_push(ddsp_server *S, int beam, const void *d_block,
                     ddsp_stream_t stream) {
  if (!S || beam < 0 || beam >= S->max_beams || !S->beams[beam].live ||
      !d_block || ((uintptr_t)d_block & 15))
    return DDSP_E_INVALID_ARG;
  ServerBeam &b = S->beams[beam];
  const int64_t j = b.pushed;
  // the slot of block j - slots is read last by the step of block j - 1
  if (j >= 1 && b.processed < j) return DDSP_E_STATE;
  DeviceGuard g(S->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (j >= 1) e = cudaStreamWaitEvent(s, step_event(*S, b.step_of[(j - 1) % 4]), 0);
  const Plan &p = S->plan->p;
  const int64_t slot = j % S->slots;
  // only the slot's columns (and the mirror's) are written
  if (e == cudaSuccess)
    e = launch_unpack_cols(d_block, S->B, p.nchan, 8, b.ring + slot * S->B,
                           S->pitch, S->B, s);
  if (e == cudaSuccess && slot == 0)   // the mirrored row tail
    e = launch_unpack_cols(d_block, S->M, p.nchan, 8, b.ring + S->R, S->pitch,
                           S->M, s);
  if (e == cudaSuccess) e = cudaEventRecord(b.ev_push[j & 1], s);
  if (e != cudaSuccess) return cuda_rc(e);
  b.push_seq[j & 1] = S->npushes++;
  b.pushed = j + 1;
  return DDSP_OK;
}

int ddsp_server_step(ddsp_server *S, float threshold, int max_beams_in_step,
                     ddsp_stream_t stream, int64_t *step_id, int *beams_out,
                     int cap, int *nbeams) {
  if (!S || !nbeams || !(threshold > 0.0f) || !isfinite(threshold) ||
      max_beams_in_step < 0)
    return DDSP_E_INVALID_ARG;
  *nbeams = 0;
  if (step_id) *step_id = -1;
  DeviceGuard g(S->device);
  cudaStream_t s = (cudaStream_t)stream;
  const Plan &p = S->plan->p;
  const int64_t id = S->nsteps;
  const int par = (int)(id & 1);
  // the staging of step id - 2 must have been read before it is rewritten
  cudaError_t e = cudaSuccess;
  if (id >= 2) e = cudaEventSynchronize(step_event(*S, id - 2));
  if (e != cudaSuccess) return cuda_rc(e);
  // beams with a block waiting, oldest push first
  std::vector<int> ready;
  for (int i = 0; i < S->max_beams; ++i) {
    const ServerBeam &b = S->beams[i];
    if (b.live && b.processed < b.pushed) ready.push_back(i);
  }
  auto seq = [&](int i) {
    const ServerBeam &b = S->beams[i];
    return b.push_seq[b.processed & 1];
  };
  std::sort(ready.begin(), ready.end(),
            [&](int a, int c) { return seq(a) < seq(c); });
  if (max_beams_in_step > 0 && (int)ready.size() > max_beams_in_step)
    ready.resize(max_beams_in_step);
  int n = 0;
  std::vector<int64_t> t0s;
  std::vector<int> members;
  for (int i : ready) {
    ServerBeam &b = S->beams[i];
    const int64_t j = b.processed;
    if ((e = cudaStreamWaitEvent(s, b.ev_push[j & 1], 0)) != cudaSuccess)
      return cuda_rc(e);
    // series slot q of its group (groups of G beam-blocks in step order)
    const int q = n % S->G;
    int32_t *series = pool_slot(*S, q);
    WsBeam &w = S->h_wsb[par][n];
    memset(&w, 0, sizeof(w));
    w.cm = b.ring;
    w.pitch = S->pitch;
    w.nsamp_out = S->B;
    w.ring = S->R;
    w.t0 = floor_mod(j * S->B - S->D16, S->R);
    t0s.push_back(w.t0);
    members.push_back(i);
    w.out_pitch = S->ncols;
    w.desc = reinterpret_cast<const int2 *>(S->tab.d_desc);
    w.relb = S->tab.d_relb;
    w.rowmap = S->tab.d_rowmap;
    w.out = series + S->C;
    w.nchan = p.nchan;
    w.n_dm_tiles = S->tab.n_dm_tiles;
    w.n_time_tiles = S->ntt;
    w.cc = S->cc;
    w.rawmax = S->rawmax;
    w.elmax = S->elmax;
    SpsBeam &q_ = S->h_sb[par][n];
    memset(&q_, 0, sizeof(q_));
    q_.series = series;
    q_.widths = p.d_widths;
    q_.m2 = b.m2;
    q_.mad4 = b.mad4;
    q_.cands = b.cands + (size_t)(j & 1) * S->cap;
    q_.count = S->d_counts + 2 * i + (j & 1);
    q_.err = S->d_err;
    q_.n = S->ncols;
    q_.L = p.norm_window;
    q_.nwin = S->nwin;
    q_.block0 = (int64_t)q * p.ndm * S->nwin;   // within its group's launch
    q_.nrep = S->B;
    q_.ndm = p.ndm;
    q_.nw = p.nwidths;
    q_.cap = S->cap;
    S->h_carry[par][n] = b.carry;
    if (beams_out && n < cap) beams_out[n] = i;
    ++n;
  }
  if (n == 0) return DDSP_OK;
  // steps run in order even if the caller moves between streams
  if (id >= 1) e = cudaStreamWaitEvent(s, step_event(*S, id - 1), 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(S->d_wsb[par], S->h_wsb[par], n * sizeof(WsBeam),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(S->d_sb[par], S->h_sb[par], n * sizeof(SpsBeam),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(S->d_carry[par], S->h_carry[par],
                        n * sizeof(int32_t *), cudaMemcpyHostToDevice, s);
  // groups of G beam-blocks, each through carry in, dedispersion, search and
  // carry out on the G series slots
  for (int g0 = 0; g0 < n && e == cudaSuccess; g0 += S->G) {
    const int gn = std::min(S->G, n - g0);
    const int64_t nitems = (int64_t)gn * S->ipb;
    if (nitems > 0x7fffffff) e = cudaErrorInvalidValue;
    if (e == cudaSuccess)
      e = launch_serve_carry(S->d_sb[par] + g0, S->d_carry[par] + g0, gn,
                             p.ndm, S->ncols, (int)S->C, true, S->d_queue, s);
    if (e == cudaSuccess && S->mode == DDSP_SERVER_INTERLEAVED) {
      e = server_dedisperse_il(*S, members.data() + g0, t0s.data() + g0, gn,
                               s);
    } else if (e == cudaSuccess) {
      e = launch_dedisperse_persistent(
          S->tile, S->d_wsb[par] + g0, nullptr, (int)nitems, S->ipb,
          S->tab.n_dm_tiles, S->d_queue, S->smem, S->d_err,
          (int)std::min<int64_t>(S->grid, nitems), s);
    }
    if (e == cudaSuccess)
      e = launch_sps_batch(S->d_sb[par] + g0, gn,
                           (int64_t)gn * p.ndm * S->nwin, threshold,
                           S->sps_smem, S->sps_cap, s);
    if (e == cudaSuccess)
      e = launch_serve_carry(S->d_sb[par] + g0, S->d_carry[par] + g0, gn,
                             p.ndm, S->ncols, (int)S->C, false, nullptr, s);
  }
  if (e == cudaSuccess) e = cudaEventRecord(step_event(*S, id), s);
  if (e != cudaSuccess) return cuda_rc(e);
  // only the last group's series are still in their slots after the step
  for (auto &b : S->beams) b.series_slot = -1;
  const int last0 = ((n - 1) / S->G) * S->G;
  for (int k = 0; k < n; ++k) {
    ServerBeam &b = S->beams[members[k]];
    b.step_of[b.processed % 4] = id;
    ++b.processed;
    if (k >= last0) b.series_slot = k % S->G;
  }
  S->nsteps = id + 1;
  if (step_id) *step_id = id;
  *nbeams = n;
  return DDSP_OK;
}

int ddsp_server_query(ddsp_server *S, int64_t step_id) {
  if (!S || step_id < 0 || step_id >= S->nsteps) return DDSP_E_INVALID_ARG;
  if (step_id < S->nsteps - kStepEvents) return 1;  // later steps were recorded
  DeviceGuard g(S->device);
  cudaError_t e = cudaEventQuery(step_event(*S, step_id));
  if (e == cudaSuccess) return 1;
  if (e == cudaErrorNotReady) return 0;
  return cuda_rc(e);
}

int ddsp_server_fetch(ddsp_server *S, int beam, int64_t block,
                      ddsp_cand *host_buf, size_t cap, size_t *n_found,
                      int64_t *t_start) {
  if (!S || beam < 0 || beam >= S->max_beams || !S->beams[beam].live ||
      !n_found || (cap > 0 && !host_buf))
    return DDSP_E_INVALID_ARG;
  ServerBeam &b = S->beams[beam];
  // the last two processed blocks keep their candidates
  if (block < 0 || block >= b.processed || block < b.processed - 2)
    return DDSP_E_STATE;
  DeviceGuard g(S->device);
  cudaError_t e = cudaEventSynchronize(step_event(*S, b.step_of[block % 4]));
  uint32_t cnt = 0;
  // copies through the plan's non-blocking copy stream: the legacy default
  // stream would also wait for the steps queued since
  if (e == cudaSuccess)
    e = copy_to_host(S->plan->p, &cnt, S->d_counts + 2 * beam + (block & 1), 4);
  if (e != cudaSuccess) return cuda_rc(e);
  const size_t stored = std::min<size_t>(cnt, S->cap);
  const size_t ncopy = std::min(stored, cap);
  if (ncopy > 0) {
    e = copy_to_host(S->plan->p, host_buf, b.cands + (size_t)(block & 1) * S->cap,
                     ncopy * sizeof(ddsp_cand));
    if (e != cudaSuccess) return cuda_rc(e);
    std::sort(host_buf, host_buf + ncopy,
              [](const ddsp_cand &a, const ddsp_cand &c) {
                return a.dm_idx != c.dm_idx ? a.dm_idx < c.dm_idx : a.t < c.t;
              });
  }
  *n_found = cnt;
  if (t_start) *t_start = block * S->B - S->D16 - S->C;
  return (cnt > ncopy) ? DDSP_E_TRUNCATED : DDSP_OK;
}

int ddsp_server_series(ddsp_server *S, int beam, int32_t **d_series,
                       int64_t *ncols) {
  if (!S || beam < 0 || beam >= S->max_beams || !S->beams[beam].live ||
      !d_series)
    return DDSP_E_INVALID_ARG;
  const int q = S->beams[beam].series_slot;
  if (q < 0) return DDSP_E_STATE;
  *d_series = pool_slot(*S, q);
  if (ncols) *ncols = S->ncols;
  return DDSP_OK;
}

int ddsp_server_check(ddsp_server *S, ddsp_stream_t stream) {
  if (!S) return DDSP_E_INVALID_ARG;
  DeviceGuard g(S->device);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_rc(e);
  int32_t v = 0;
  e = cudaMemcpy(&v, S->d_err, 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_rc(e);
  if (v != kErrNone) {
    cudaMemset(S->d_err, 0, 4);
    return v == kErrRange ? DDSP_E_RANGE : DDSP_E_TIMEOUT;
  }
  return DDSP_OK;
}

}  // extern "C"
