// batch.cu -- many beams (plans) of uneven shape dedispersed by one
// persistent launch and searched by one batched launch, optionally replayed
// from a captured CUDA graph; tile autotuner.
#include <math.h>

#include <algorithm>
#include <new>
#include <vector>

#include "host.h"
#include "ws_item.cuh"

using namespace ddsp;

struct ddsp_batch {
  int device = 0;
  int nbeams = 0;
  std::vector<ddsp_plan *> plans;
  std::vector<int64_t> nin, nout, pitch;
  std::vector<DedispTables> tabs;  // per beam, for the common tile
  DedispTile tile;                 // chan_chunk = the per-beam upper limit
  std::vector<int> cc;             // per-beam channel chunk
  int grid = 0;
  size_t smem = 0;
  // device buffers
  std::vector<int32_t *> d_out;     // per-beam series (caller's or own_out)
  std::vector<int32_t *> own_out;   // the ones the batch allocated
  uint8_t *d_cm = nullptr;
  size_t cm_bytes = 0;
  std::vector<size_t> cm_off;
  WsBeam *d_wsb = nullptr;
  int4 *d_items = nullptr;
  int nitems = 0;
  std::vector<int4> items;         // host copy of the work list
  int *d_queue = nullptr;
  SpsBeam *d_sb = nullptr;
  int64_t sps_blocks = 0;
  size_t sps_smem = 0;
  uint32_t **d_counts = nullptr;
  int32_t *d_err = nullptr;
  // graph
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  bool graph_ok = false;
  float graph_thr = 0.0f;
  bool ran_direct = false;
};

namespace {

void batch_free_graph(ddsp_batch &B) {
  if (B.gexec) cudaGraphExecDestroy(B.gexec);
  if (B.graph) cudaGraphDestroy(B.graph);
  B.gexec = nullptr;
  B.graph = nullptr;
  B.graph_ok = false;
}

void batch_release(ddsp_batch &B) {
  batch_free_graph(B);
  if (B.cap_stream) cudaStreamDestroy(B.cap_stream);
  for (auto &t : B.tabs) free_tables(t);
  for (auto p : B.own_out) cudaFree(p);
  cudaFree(B.d_cm);
  cudaFree(B.d_wsb);
  cudaFree(B.d_items);
  cudaFree(B.d_queue);
  cudaFree(B.d_sb);
  cudaFree(B.d_counts);
  cudaFree(B.d_err);
}

constexpr int64_t kBatchMaxTimeTile = 4 * 32 * kElemPerThread * 8;

// One beam's warp-specialised layout for tile t: its buffer extents and the
// largest channel chunk <= t.chan_chunk whose layout fits `budget` bytes
// (0 if even one channel does not fit).
struct BeamLayout {
  int cc = 0, rawmax = 0, elmax = 0;
  size_t smem = 0;
};

BeamLayout beam_layout(const Plan &p, const DedispTile &t, size_t budget) {
  BeamLayout b;
  dedisp_buffer_sizes(t, span_for(p, t.dm_tile()), 8, &b.rawmax, &b.elmax);
  for (int cc = t.chan_chunk; cc >= 1; --cc) {
    const size_t sm =
        dedisp_ws_smem_bytes(cc, t.dm_tile(), b.rawmax, b.elmax, t.nbuf);
    if (sm <= budget) {
      b.cc = cc;
      b.smem = sm;
      return b;
    }
  }
  return b;
}

// Per-beam layouts of tile t: every beam within the two-blocks-per-SM
// budget if they all fit it, else within the one-block budget.  The launch's
// shared memory is the largest of them.
bool batch_layout(const ddsp_batch &B, const DedispTile &t,
                  std::vector<BeamLayout> *out, size_t *smem) {
  for (size_t budget : {kSmemBudgetTwoBlocks, kSmemBudgetOneBlock}) {
    out->assign(B.nbeams, BeamLayout{});
    *smem = 0;
    bool all = true;
    for (int b = 0; b < B.nbeams && all; ++b) {
      (*out)[b] = beam_layout(B.plans[b]->p, t, budget);
      all = (*out)[b].cc > 0;
      *smem = std::max(*smem, (*out)[b].smem);
    }
    if (all) return true;
  }
  return false;
}

// Build per-beam tables, channel-major workspaces and the dedispersion work
// list for tile t; the tile's time tile fixes every beam's pitch.
int batch_apply_tile(ddsp_batch &B, const DedispTile &t) {
  std::vector<BeamLayout> lay;
  size_t smem;
  if (!dedisp_tile_supported(t, 8) || !(t.flags & kTileWarpSpecialized) ||
      !batch_layout(B, t, &lay, &smem))
    return DDSP_E_INVALID_ARG;
  batch_free_graph(B);
  cudaDeviceSynchronize();
  const int TT = dedisp_time_tile(t, 8);
  if (TT > kBatchMaxTimeTile) return DDSP_E_INVALID_ARG;
  B.tabs.resize(B.nbeams);
  B.pitch.resize(B.nbeams);
  B.cm_off.resize(B.nbeams);
  size_t cm_bytes = 0;
  for (int b = 0; b < B.nbeams; ++b) {
    const Plan &p = B.plans[b]->p;
    int rc = build_tables_for(p, t, B.tabs[b]);
    if (rc != DDSP_OK) return rc;
    // pitch sized for the largest time tile of any shape, so the ingested
    // rows stay valid when the tile changes
    B.pitch[b] = round_up(round_up(B.nout[b], kBatchMaxTimeTile) +
                              p.max_delay + 64, 128);
    B.cm_off[b] = cm_bytes;
    cm_bytes += ((size_t)p.nchan * B.pitch[b] + 255) & ~(size_t)255;
  }
  cudaError_t e = cudaSuccess;
  if (cm_bytes > B.cm_bytes) {  // the pool only grows (its contents stay)
    uint8_t *nw = nullptr;
    if ((e = cudaMalloc(&nw, cm_bytes)) != cudaSuccess) return cuda_rc(e);
    cudaFree(B.d_cm);
    B.d_cm = nw;
    B.cm_bytes = cm_bytes;
  }
  // descriptors
  std::vector<WsBeam> wsb(B.nbeams);
  std::vector<int4> items;
  for (int b = 0; b < B.nbeams; ++b) {
    const Plan &p = B.plans[b]->p;
    WsBeam &w = wsb[b];
    w.cm = B.d_cm + B.cm_off[b];
    w.pitch = B.pitch[b];
    w.nsamp_out = B.nout[b];
    w.ring = 0;
    w.t0 = 0;
    w.out_pitch = B.nout[b];
    w.desc = reinterpret_cast<const int2 *>(B.tabs[b].d_desc);
    w.relb = B.tabs[b].d_relb;
    w.rowmap = B.tabs[b].d_rowmap;
    w.out = B.d_out[b];
    w.nchan = p.nchan;
    w.n_dm_tiles = B.tabs[b].n_dm_tiles;
    w.n_time_tiles = (int)((B.nout[b] + TT - 1) / TT);
    w.cc = lay[b].cc;
    w.rawmax = lay[b].rawmax;
    w.elmax = lay[b].elmax;
    // DM tiles innermost: consecutive items stage overlapping windows of
    // one time tile, which L2 then serves
    for (int tt = 0; tt < w.n_time_tiles; ++tt)
      for (int g = 0; g < w.n_dm_tiles; ++g)
        items.push_back(make_int4(b, g, tt, p.nchan));
  }
  // the costliest items (most channels) first, so the tail is short
  std::stable_sort(items.begin(), items.end(),
                   [](const int4 &a, const int4 &b) { return a.w > b.w; });
  cudaFree(B.d_wsb);
  cudaFree(B.d_items);
  B.d_wsb = nullptr;
  B.d_items = nullptr;
  if ((e = cudaMalloc(&B.d_wsb, wsb.size() * sizeof(WsBeam))) != cudaSuccess ||
      (e = cudaMalloc(&B.d_items, items.size() * sizeof(int4))) != cudaSuccess)
    return cuda_rc(e);
  cudaMemcpy(B.d_wsb, wsb.data(), wsb.size() * sizeof(WsBeam),
             cudaMemcpyHostToDevice);
  e = cudaMemcpy(B.d_items, items.data(), items.size() * sizeof(int4),
                 cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_rc(e);
  B.nitems = (int)items.size();
  B.items.swap(items);
  B.tile = t;
  B.cc.resize(B.nbeams);
  for (int b = 0; b < B.nbeams; ++b) B.cc[b] = lay[b].cc;
  B.smem = smem;
  int per_sm = persistent_blocks_per_sm(t, smem);
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, B.device);
  if (per_sm <= 0 || nsm <= 0) return DDSP_E_INVALID_ARG;
  B.grid = std::min(per_sm * nsm, std::max(1, B.nitems));
  return DDSP_OK;
}

// Candidate tiles; chan_chunk is the per-beam upper limit.
const DedispTile kBatchTiles[] = {
    // {wt, wd, rd, chan_chunk, nbuf, flags}
    {4, 2, 8, 8, 2, kTileWarpSpecialized}, {4, 2, 8, 6, 2, kTileWarpSpecialized},
    {4, 2, 8, 4, 2, kTileWarpSpecialized}, {4, 2, 8, 4, 4, kTileWarpSpecialized},
    {8, 1, 8, 6, 2, kTileWarpSpecialized}, {8, 1, 8, 4, 2, kTileWarpSpecialized},
    {2, 4, 8, 8, 2, kTileWarpSpecialized}, {4, 2, 4, 8, 2, kTileWarpSpecialized},
    {8, 1, 4, 6, 2, kTileWarpSpecialized}, {8, 1, 4, 4, 4, kTileWarpSpecialized}};
constexpr int kNumBatchTiles = sizeof(kBatchTiles) / sizeof(kBatchTiles[0]);
constexpr size_t kAutotuneStride = 16;

int batch_enqueue(ddsp_batch &B, float thr, cudaStream_t s) {
  cudaError_t e = launch_batch_reset(B.d_queue, B.d_counts, B.nbeams, s);
  if (e == cudaSuccess)
    e = launch_dedisperse_persistent(B.tile, B.d_wsb, B.d_items, B.nitems, 0,
                                     0, B.d_queue, B.smem, B.d_err, B.grid, s);
  if (e == cudaSuccess)
    e = launch_sps_batch(B.d_sb, B.nbeams, B.sps_blocks, thr, B.sps_smem, s);
  return cuda_rc(e);
}

}  // namespace

extern "C" {

int ddsp_batch_create(ddsp_batch **out, ddsp_plan *const *plans, int nbeams,
                      const int64_t *nsamp_in, int32_t *const *d_series) {
  if (!out || !plans || !nsamp_in || nbeams <= 0) return DDSP_E_INVALID_ARG;
  *out = nullptr;
  for (int b = 0; b < nbeams; ++b) {
    if (!plans[b]) return DDSP_E_INVALID_ARG;
    const Plan &p = plans[b]->p;
    if (p.nbits != 8 || p.nchan % 16 != 0) return DDSP_E_INVALID_ARG;
    if (nsamp_in[b] - p.max_delay <= 0) return DDSP_E_SHAPE;
    if (p.device != plans[0]->p.device) return DDSP_E_INVALID_ARG;
    int64_t nwin;
    if (search_windows(p, nsamp_in[b] - p.max_delay, &nwin) != DDSP_OK)
      return DDSP_E_SHAPE;
  }
  ddsp_batch *B = new (std::nothrow) ddsp_batch;
  if (!B) return DDSP_E_NOMEM;
  B->device = plans[0]->p.device;
  DeviceGuard g(B->device);
  B->nbeams = nbeams;
  B->plans.assign(plans, plans + nbeams);
  B->nin.assign(nsamp_in, nsamp_in + nbeams);
  B->nout.resize(nbeams);
  B->d_out.assign(nbeams, nullptr);
  int rc = DDSP_OK;
  cudaError_t e = cudaSuccess;
  std::vector<SpsBeam> sb(nbeams);
  std::vector<uint32_t *> counts(nbeams);
  int64_t sblocks = 0;
  int64_t maxlen_all = 0;
  int wmax_all = 1;
  for (int b = 0; b < nbeams && rc == DDSP_OK; ++b) {
    Plan &p = plans[b]->p;
    const int64_t nout = nsamp_in[b] - p.max_delay;
    B->nout[b] = nout;
    if (d_series && d_series[b]) {
      B->d_out[b] = d_series[b];
    } else {
      if ((e = cudaMalloc(&B->d_out[b], (size_t)p.ndm * nout * 4)) != cudaSuccess) {
        rc = cuda_rc(e);
        break;
      }
      B->own_out.push_back(B->d_out[b]);
    }
    int64_t nwin;
    search_windows(p, nout, &nwin);
    rc = ensure_stats(p, (size_t)nwin * p.ndm);
    if (rc != DDSP_OK) break;
    const int64_t L = p.norm_window;
    const int64_t maxlen =
        (L <= 0 || nwin == 1) ? nout : std::max(L, nout - (nwin - 1) * L);
    maxlen_all = std::max(maxlen_all, maxlen);
    wmax_all = std::max(wmax_all, p.widths.back());
    SpsBeam &s = sb[b];
    s.series = B->d_out[b];
    s.widths = p.d_widths;
    s.m2 = p.d_m2;
    s.mad4 = p.d_mad4;
    s.cands = p.d_cands;
    s.count = p.d_count;
    s.err = p.d_err;
    s.n = nout;
    s.nrep = nout;
    s.L = L;
    s.nwin = nwin;
    s.block0 = sblocks;
    s.ndm = p.ndm;
    s.nw = p.nwidths;
    s.cap = (uint32_t)p.cand_capacity;
    sblocks += nwin * p.ndm;
    counts[b] = p.d_count;
  }
  if (rc == DDSP_OK) {
    B->sps_blocks = sblocks;
    B->sps_smem = sps_smem_bytes(maxlen_all, wmax_all);
    if ((e = cudaMalloc(&B->d_sb, sb.size() * sizeof(SpsBeam))) != cudaSuccess ||
        (e = cudaMalloc(&B->d_counts, counts.size() * sizeof(uint32_t *))) != cudaSuccess ||
        (e = cudaMalloc(&B->d_queue, sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&B->d_err, sizeof(int32_t))) != cudaSuccess)
      rc = cuda_rc(e);
  }
  if (rc == DDSP_OK) {
    cudaMemcpy(B->d_sb, sb.data(), sb.size() * sizeof(SpsBeam), cudaMemcpyHostToDevice);
    cudaMemcpy(B->d_counts, counts.data(), counts.size() * sizeof(uint32_t *),
               cudaMemcpyHostToDevice);
    cudaMemset(B->d_err, 0, sizeof(int32_t));
    rc = DDSP_E_INVALID_ARG;  // unless some tile fits
    for (int i = 0; i < kNumBatchTiles && rc != DDSP_OK; ++i)
      rc = batch_apply_tile(*B, kBatchTiles[i]);
  }
  if (rc == DDSP_OK &&
      cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    rc = DDSP_E_CUDA;
  if (rc != DDSP_OK) {
    batch_release(*B);
    delete B;
    return rc;
  }
  *out = B;
  return DDSP_OK;
}

void ddsp_batch_destroy(ddsp_batch *B) {
  if (!B) return;
  DeviceGuard g(B->device);
  cudaDeviceSynchronize();
  batch_release(*B);
  delete B;
}

int ddsp_batch_input(ddsp_batch *B, int beam, void **d_cm, int64_t *pitch,
                     int64_t *nsamp_in) {
  if (!B || beam < 0 || beam >= B->nbeams || !d_cm) return DDSP_E_INVALID_ARG;
  *d_cm = B->d_cm + B->cm_off[beam];
  if (pitch) *pitch = B->pitch[beam];
  if (nsamp_in) *nsamp_in = B->nin[beam];
  return DDSP_OK;
}

int ddsp_batch_ingest(ddsp_batch *B, int beam, const void *d_in,
                      ddsp_stream_t stream) {
  if (!B || beam < 0 || beam >= B->nbeams || !d_in || ((uintptr_t)d_in & 15))
    return DDSP_E_INVALID_ARG;
  DeviceGuard g(B->device);
  const Plan &p = B->plans[beam]->p;
  return cuda_rc(launch_unpack(d_in, B->nin[beam], p.nchan, 8,
                               B->d_cm + B->cm_off[beam], B->pitch[beam],
                               (cudaStream_t)stream));
}

int ddsp_batch_series(ddsp_batch *B, int beam, int32_t **d_series,
                      int64_t *nsamp_out) {
  if (!B || beam < 0 || beam >= B->nbeams || !d_series) return DDSP_E_INVALID_ARG;
  *d_series = B->d_out[beam];
  if (nsamp_out) *nsamp_out = B->nout[beam];
  return DDSP_OK;
}

int ddsp_batch_set_tile(ddsp_batch *B, int dm_tile, int dm_per_thread,
                        int chan_chunk, int stages) {
  if (!B || dm_per_thread <= 0 || dm_tile % dm_per_thread) return DDSP_E_INVALID_ARG;
  DeviceGuard g(B->device);
  DedispTile t;
  t.rd = dm_per_thread;
  t.wd = dm_tile / dm_per_thread;
  if (t.wd <= 0 || (kThreads / 32) % t.wd) return DDSP_E_INVALID_ARG;
  t.wt = (kThreads / 32) / t.wd;
  t.chan_chunk = chan_chunk;
  t.nbuf = stages;
  t.flags = kTileWarpSpecialized;
  return batch_apply_tile(*B, t);
}

int ddsp_batch_get_beam_chunk(const ddsp_batch *B, int beam, int *chan_chunk) {
  if (!B || beam < 0 || beam >= B->nbeams || !chan_chunk)
    return DDSP_E_INVALID_ARG;
  *chan_chunk = B->cc[beam];
  return DDSP_OK;
}

int ddsp_batch_get_tile(const ddsp_batch *B, int *dm_tile, int *dm_per_thread,
                        int *time_tile, int *chan_chunk, int *stages,
                        int *grid) {
  if (!B) return DDSP_E_INVALID_ARG;
  if (dm_tile) *dm_tile = B->tile.dm_tile();
  if (dm_per_thread) *dm_per_thread = B->tile.rd;
  if (time_tile) *time_tile = dedisp_time_tile(B->tile, 8);
  if (chan_chunk) *chan_chunk = B->tile.chan_chunk;
  if (stages) *stages = B->tile.nbuf;
  if (grid) *grid = B->grid;
  return DDSP_OK;
}

int ddsp_batch_run(ddsp_batch *B, float threshold, int use_graph,
                   ddsp_stream_t stream) {
  if (!B || !(threshold > 0.0f) || !isfinite(threshold)) return DDSP_E_INVALID_ARG;
  DeviceGuard g(B->device);
  cudaStream_t s = (cudaStream_t)stream;
  int rc;
  if (!use_graph || !B->ran_direct) {
    // the first run is direct: it also sets the kernels' shared-memory
    // limits, which must not happen during a capture
    rc = batch_enqueue(*B, threshold, s);
    if (rc != DDSP_OK) return rc;
    B->ran_direct = true;
  } else {
    if (!B->graph_ok || B->graph_thr != threshold) {
      batch_free_graph(*B);
      cudaError_t e = cudaStreamBeginCapture(B->cap_stream,
                                             cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_rc(e);
      rc = batch_enqueue(*B, threshold, B->cap_stream);
      e = cudaStreamEndCapture(B->cap_stream, &B->graph);
      if (rc != DDSP_OK) return rc;
      if (e != cudaSuccess) return cuda_rc(e);
      e = cudaGraphInstantiate(&B->gexec, B->graph, 0);
      if (e != cudaSuccess) return cuda_rc(e);
      B->graph_ok = true;
      B->graph_thr = threshold;
    }
    cudaError_t e = cudaGraphLaunch(B->gexec, s);
    if (e != cudaSuccess) return cuda_rc(e);
  }
  for (int b = 0; b < B->nbeams; ++b) {
    Plan &p = B->plans[b]->p;
    int64_t nwin;
    search_windows(p, B->nout[b], &nwin);
    p.searched = true;
    p.last_stream = s;
    p.last_nwin = nwin;
  }
  return DDSP_OK;
}

int ddsp_batch_check(ddsp_batch *B, ddsp_stream_t stream) {
  if (!B) return DDSP_E_INVALID_ARG;
  DeviceGuard g(B->device);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_rc(e);
  int32_t v = 0;
  e = cudaMemcpy(&v, B->d_err, 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_rc(e);
  if (v != kErrNone) {
    cudaMemset(B->d_err, 0, 4);
    return DDSP_E_TIMEOUT;
  }
  for (auto h : B->plans) {
    int rc = read_err(h->p);
    if (rc != DDSP_OK) return rc;
  }
  return DDSP_OK;
}

int ddsp_batch_autotune(ddsp_batch *B, int reps, ddsp_stream_t stream,
                        float *ms_out, int cap, int *ntried, int *best) {
  if (!B || reps <= 0) return DDSP_E_INVALID_ARG;
  DeviceGuard g(B->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int tried = 0, besti = -1;
  float bestms = 1e30f;
  int4 *d_sample = nullptr;
  size_t sample_cap = 0;
  for (int i = 0; i < kNumBatchTiles; ++i) {
    float ms = -1.0f;
    if (batch_apply_tile(*B, kBatchTiles[i]) == DDSP_OK) {
      // every kAutotuneStride-th item of the cost-ordered work list: the
      // same share of every beam's work for each candidate
      std::vector<int4> sample;
      for (size_t k = 0; k < B->items.size(); k += kAutotuneStride)
        sample.push_back(B->items[k]);
      cudaError_t e = cudaSuccess;
      if (sample.size() > sample_cap) {
        cudaFree(d_sample);
        d_sample = nullptr;
        sample_cap = 0;
        e = cudaMalloc(&d_sample, sample.size() * sizeof(int4));
        if (e == cudaSuccess) sample_cap = sample.size();
      }
      if (e == cudaSuccess)
        e = cudaMemcpy(d_sample, sample.data(), sample.size() * sizeof(int4),
                       cudaMemcpyHostToDevice);
      const int grid = std::min(B->grid, (int)sample.size());
      float best_rep = 1e30f;
      for (int r = 0; r <= reps && e == cudaSuccess; ++r) {
        launch_batch_reset(B->d_queue, B->d_counts, B->nbeams, s);
        cudaEventRecord(e0, s);
        e = launch_dedisperse_persistent(B->tile, B->d_wsb, d_sample,
                                         (int)sample.size(), 0, 0, B->d_queue,
                                         B->smem, B->d_err, grid, s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float t = 0;
        cudaEventElapsedTime(&t, e0, e1);
        if (r > 0) best_rep = std::min(best_rep, t);  // first run warms up
      }
      if (e == cudaSuccess)
        ms = best_rep * (float)B->items.size() / (float)sample.size();
      if (ms > 0 && ms < bestms) {
        bestms = ms;
        besti = i;
      }
    }
    if (ms_out && i < cap) ms_out[i] = ms;
    ++tried;
  }
  cudaFree(d_sample);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (ntried) *ntried = tried;
  if (best) *best = besti;
  if (besti < 0) return DDSP_E_INVALID_ARG;
  B->ran_direct = false;
  return batch_apply_tile(*B, kBatchTiles[besti]);
}

}  // extern "C"
