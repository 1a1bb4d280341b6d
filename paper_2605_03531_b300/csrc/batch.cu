// batch.cu -- many beams (plans) of uneven shape dedispersed by persistent
// launches (one per tile group: the main shape, and a narrower-DM shape for
// beams whose delay spans make the main one stage little and relayout a lot)
// or, in the per-beam mode, beam after beam by the interleaved kernel
// (each beam's rows interleaved into one shared staging area first: the
// interleaved rows of all beams at once would not fit in HBM), and
// searched by one batched launch, optionally replayed from a captured CUDA
// graph; tile and mode autotuner.
#include <math.h>

#include <algorithm>
#include <new>
#include <vector>

#include "host.h"
#include "ws_item.cuh"

using namespace ddsp;

namespace {
constexpr int kMaxGroups = 2;

// Beams that share one persistent launch (one tile shape).
struct BatchGroup {
  DedispTile tile;                 // chan_chunk = the per-beam upper limit
  std::vector<int> beams;          // batch beam indices
  WsBeam *d_wsb = nullptr;         // [beams.size()]
  int4 *d_items = nullptr;         // {group-local beam, DM tile, time tile, cost}
  std::vector<int4> items;         // host copy of the work list
  int nitems = 0, grid = 0;
  size_t smem = 0;
};
}  // namespace

struct ddsp_batch {
  int device = 0;
  int nbeams = 0;
  std::vector<ddsp_plan *> plans;
  std::vector<int64_t> nin, nout, pitch;
  std::vector<DedispTables> tabs;  // per beam, for its group's tile
  DedispTile tile;                 // the main group's tile
  std::vector<int> cc;             // per-beam channel chunk
  std::vector<int> group_of;       // per-beam group
  std::vector<BatchGroup> groups;
  // largest delay spread inside a DM tile of 2^k trials, per beam (-1: not
  // computed yet)
  mutable std::vector<std::vector<int>> span_cache;
  // device buffers
  std::vector<int32_t *> d_out;     // per-beam series (caller's or own_out)
  std::vector<int32_t *> own_out;   // the ones the batch allocated
  uint8_t *d_cm = nullptr;
  size_t cm_bytes = 0;
  std::vector<size_t> cm_off;
  int *d_queue = nullptr;          // [kMaxGroups] work-queue counters
  SpsBeam *d_sb = nullptr;
  int64_t sps_blocks = 0;
  size_t sps_smem = 0;
  int64_t sps_cap = 0;
  uint32_t **d_counts = nullptr;
  int32_t *d_err = nullptr;
  // graph
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  bool graph_ok = false;
  float graph_thr = 0.0f;
  bool ran_direct = false;
  // per-beam interleaved mode (DDSP_BATCH_PER_BEAM)
  int mode = DDSP_BATCH_PERSISTENT;
  std::vector<DedispTile> il_tile;   // per beam: its plan's default tile
  std::vector<DedispTables> il_tabs; // per beam, for il_tile
  void *d_il = nullptr;              // shared staging rows (largest beam)
  size_t il_bytes = 0;
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
  for (auto &t : B.il_tabs) free_tables(t);
  cudaFree(B.d_il);
  for (auto p : B.own_out) cudaFree(p);
  cudaFree(B.d_cm);
  for (auto &g : B.groups) {
    cudaFree(g.d_wsb);
    cudaFree(g.d_items);
  }
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

int beam_span(const ddsp_batch &B, int b, int dt) {
  int k = 0;
  while ((1 << k) < dt) ++k;
  auto &c = B.span_cache;
  if (c.size() != (size_t)B.nbeams) c.assign(B.nbeams, std::vector<int>(8, -1));
  if ((1 << k) != dt || k >= 8) return span_for(B.plans[b]->p, dt);
  if (c[b][k] < 0) c[b][k] = span_for(B.plans[b]->p, dt);
  return c[b][k];
}

BeamLayout beam_layout(const ddsp_batch &B, int beam, const DedispTile &t,
                       size_t budget) {
  BeamLayout b;
  dedisp_buffer_sizes(t, beam_span(B, beam, t.dm_tile()), 8, &b.rawmax,
                      &b.elmax);
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

// Relayouted elements per consumed word of a beam under tile t:
// (S + span) / (DT * S), S the element segment, span the largest delay
// spread inside a DM tile.  Large values mean the producers' relayout, not
// the accumulation, sets the pace.
double relayout_ratio(const ddsp_batch &B, int beam, const DedispTile &t) {
  const double S = 32.0 * kElemPerThread * t.wt;
  return (S + beam_span(B, beam, t.dm_tile())) / (t.dm_tile() * S);
}

// Narrower-DM shapes for the second group.
const DedispTile kFallbackTiles[] = {
    {8, 1, 4, 8, 2, kTileWarpSpecialized}, {8, 1, 8, 8, 2, kTileWarpSpecialized},
    {4, 2, 4, 8, 2, kTileWarpSpecialized}};

// Per-beam layouts of the group's beams under tile t: all within the
// two-blocks-per-SM budget if they fit it, else within the one-block budget.
bool group_layout(const ddsp_batch &B, const DedispTile &t,
                  const std::vector<int> &beams, std::vector<BeamLayout> *out,
                  size_t *smem) {
  for (size_t budget : {kSmemBudgetTwoBlocks, kSmemBudgetOneBlock}) {
    out->assign(beams.size(), BeamLayout{});
    *smem = 0;
    bool all = true;
    for (size_t i = 0; i < beams.size() && all; ++i) {
      (*out)[i] = beam_layout(B, beams[i], t, budget);
      all = (*out)[i].cc > 0;
      *smem = std::max(*smem, (*out)[i].smem);
    }
    if (all) return true;
  }
  return false;
}

// Split the beams between main tile t and (possibly) one fallback shape: a
// beam moves to the fallback if the main shape cannot hold it, stages fewer
// than 2 of its channels per chunk (when the chunk limit allows 2) or the
// fallback relayouts 30 % less per consumed word;
// the fallback shape is the one with the lowest adds-weighted relayout.
void choose_groups(const ddsp_batch &B, const DedispTile &t,
                   std::vector<int> *main_beams, std::vector<int> *fb_beams,
                   DedispTile *fb_tile) {
  std::vector<double> rmain(B.nbeams), adds(B.nbeams);
  std::vector<int> ccmain(B.nbeams);
  std::vector<char> nomain(B.nbeams);   // fits the main shape under no budget
  bool main_ok = true;
  for (int b = 0; b < B.nbeams; ++b) {
    const Plan &p = B.plans[b]->p;
    rmain[b] = relayout_ratio(B, b, t);
    ccmain[b] = beam_layout(B, b, t, kSmemBudgetTwoBlocks).cc;
    nomain[b] = ccmain[b] == 0 && beam_layout(B, b, t, kSmemBudgetOneBlock).cc == 0;
    main_ok = main_ok && !nomain[b];
    adds[b] = (double)p.nchan * p.ndm * B.nout[b];
  }
  double best = 0;
  for (int b = 0; b < B.nbeams; ++b) best += adds[b] * rmain[b];
  if (!main_ok) best = 1e300;
  main_beams->clear();
  for (int b = 0; b < B.nbeams; ++b) main_beams->push_back(b);
  fb_beams->clear();
  for (const DedispTile &f : kFallbackTiles) {
    if (!dedisp_tile_supported(f, 8) || dedisp_time_tile(f, 8) > kBatchMaxTimeTile)
      continue;
    std::vector<int> mb, fbb;
    double cost = 0;
    bool feasible = true;
    for (int b = 0; b < B.nbeams && feasible; ++b) {
      const double rf = relayout_ratio(B, b, f);
      const bool fits = beam_layout(B, b, f, kSmemBudgetTwoBlocks).cc > 0 ||
                        beam_layout(B, b, f, kSmemBudgetOneBlock).cc > 0;
      const bool move = fits && (nomain[b] || ccmain[b] < std::min(2, t.chan_chunk) ||
                                 rf < 0.7 * rmain[b]);
      feasible = move || !nomain[b];
      (move ? fbb : mb).push_back(b);
      cost += adds[b] * (move ? rf : rmain[b]);
    }
    if (feasible && !fbb.empty() && !mb.empty() && cost < 0.97 * best) {
      best = cost;
      *main_beams = mb;
      *fb_beams = fbb;
      *fb_tile = f;
    }
  }
}

// Build one group: per-beam tables for its tile, descriptors and the
// cost-ordered work list (uploaded).
int build_group(ddsp_batch &B, BatchGroup &G, const DedispTile &t,
                const std::vector<int> &beams) {
  std::vector<BeamLayout> lay;
  size_t smem;
  if (!group_layout(B, t, beams, &lay, &smem)) return DDSP_E_INVALID_ARG;
  const int TT = dedisp_time_tile(t, 8);
  std::vector<WsBeam> wsb(beams.size());
  std::vector<int4> items;
  for (size_t i = 0; i < beams.size(); ++i) {
    const int b = beams[i];
    const Plan &p = B.plans[b]->p;
    int rc = build_tables_for(p, t, B.tabs[b]);
    if (rc != DDSP_OK) return rc;
    WsBeam &w = wsb[i];
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
    w.cc = lay[i].cc;
    w.rawmax = lay[i].rawmax;
    w.elmax = lay[i].elmax;
    B.cc[b] = lay[i].cc;
    // DM tiles innermost: consecutive items stage overlapping windows of
    // one time tile, which L2 then serves
    for (int tt = 0; tt < w.n_time_tiles; ++tt)
      for (int g = 0; g < w.n_dm_tiles; ++g)
        items.push_back(make_int4((int)i, g, tt, p.nchan));
  }
  // the costliest items (most channels) first, so the tail is short
  std::stable_sort(items.begin(), items.end(),
                   [](const int4 &a, const int4 &b) { return a.w > b.w; });
  cudaError_t e;
  if ((e = cudaMalloc(&G.d_wsb, wsb.size() * sizeof(WsBeam))) != cudaSuccess ||
      (e = cudaMalloc(&G.d_items, items.size() * sizeof(int4))) != cudaSuccess)
    return cuda_rc(e);
  cudaMemcpy(G.d_wsb, wsb.data(), wsb.size() * sizeof(WsBeam),
             cudaMemcpyHostToDevice);
  e = cudaMemcpy(G.d_items, items.data(), items.size() * sizeof(int4),
                 cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_rc(e);
  G.tile = t;
  G.beams = beams;
  G.nitems = (int)items.size();
  G.items.swap(items);
  G.smem = smem;
  const int per_sm = persistent_blocks_per_sm(t, smem);
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, B.device);
  if (per_sm <= 0 || nsm <= 0) return DDSP_E_INVALID_ARG;
  G.grid = std::min(per_sm * nsm, std::max(1, G.nitems));
  return DDSP_OK;
}

// Apply main tile t: split the beams into groups, size the channel-major
// pool (pitches fit every time tile) and build each group.
int batch_apply_tile(ddsp_batch &B, const DedispTile &t) {
  if (!dedisp_tile_supported(t, 8) || !(t.flags & kTileWarpSpecialized) ||
      dedisp_time_tile(t, 8) > kBatchMaxTimeTile)
    return DDSP_E_INVALID_ARG;
  std::vector<int> mb, fbb;
  DedispTile ft;
  choose_groups(B, t, &mb, &fbb, &ft);
  {
    std::vector<BeamLayout> lay;
    size_t sm;
    if (!group_layout(B, t, mb, &lay, &sm)) return DDSP_E_INVALID_ARG;
  }
  batch_free_graph(B);
  cudaDeviceSynchronize();
  B.tabs.resize(B.nbeams);
  B.pitch.resize(B.nbeams);
  B.cm_off.resize(B.nbeams);
  B.cc.assign(B.nbeams, 0);
  B.group_of.assign(B.nbeams, 0);
  size_t cm_bytes = 0;
  for (int b = 0; b < B.nbeams; ++b) {
    const Plan &p = B.plans[b]->p;
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
  for (auto &g : B.groups) {
    cudaFree(g.d_wsb);
    cudaFree(g.d_items);
  }
  B.groups.assign(fbb.empty() ? 1 : 2, BatchGroup{});
  int rc = build_group(B, B.groups[0], t, mb);
  if (rc == DDSP_OK && !fbb.empty()) {
    rc = build_group(B, B.groups[1], ft, fbb);
    for (int b : fbb) B.group_of[b] = 1;
  }
  if (rc != DDSP_OK) return rc;
  B.tile = t;
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

// The interleaved tile a beam runs with in the per-beam mode, within the
// time tiles the pool's pitch allows.
DedispTile il_tile_for(const ddsp_batch &B, int b) {
  return fit_interleaved_tile(
      [](int tt) { return tt <= kBatchMaxTimeTile; },
      [&](int dt) { return beam_span(B, b, dt); });
}

// Per-beam interleaved mode: every beam needs an interleaved tile
// (il_tile_for); one staging area, sized for the largest beam, serves the
// beams in turn (stream order).  Builds the tables once.
int batch_setup_il(ddsp_batch &B) {
  if (!B.il_tabs.empty()) return DDSP_OK;
  std::vector<DedispTile> tiles(B.nbeams);
  size_t bytes = 0;
  for (int b = 0; b < B.nbeams; ++b) {
    const Plan &p = B.plans[b]->p;
    const DedispTile t = il_tile_for(B, b);
    if (t.wt == 0) return DDSP_E_INVALID_ARG;
    tiles[b] = t;
    bytes = std::max(bytes, (size_t)p.nchan * B.pitch[b] * 4);
  }
  std::vector<DedispTables> tabs(B.nbeams);
  int rc = DDSP_OK;
  for (int b = 0; b < B.nbeams && rc == DDSP_OK; ++b)
    rc = build_tables_for(B.plans[b]->p, tiles[b], tabs[b]);
  void *d_il = nullptr;
  if (rc == DDSP_OK) {
    cudaError_t e = cudaMalloc(&d_il, bytes);
    if (e != cudaSuccess) rc = cuda_rc(e);
  }
  if (rc != DDSP_OK) {
    for (auto &t : tabs) free_tables(t);
    return rc;
  }
  B.il_tile.swap(tiles);
  B.il_tabs.swap(tabs);
  B.d_il = d_il;
  B.il_bytes = bytes;
  return DDSP_OK;
}

// Every beam's interleave + dedispersion, in turn, into its series.
cudaError_t batch_dedisperse_per_beam(ddsp_batch &B, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < B.nbeams && e == cudaSuccess; ++b) {
    const Plan &p = B.plans[b]->p;
    IlLaunch v;
    v.tile = B.il_tile[b];
    v.tab = &B.il_tabs[b];
    v.nchan = p.nchan;
    v.nbits = 8;
    v.d_err = B.d_err;
    v.d_il = B.d_il;
    // the pool's rows hold the block, zeros past it (ingest) or whatever
    // the caller wrote; samples past N_in reach no stored output
    e = launch_interleave(v, B.d_cm + B.cm_off[b], B.pitch[b], B.nin[b],
                          B.pitch[b], s);
    if (e == cudaSuccess)
      e = launch_dedisperse_il(v, B.pitch[b], B.nout[b], B.d_out[b], s);
  }
  return e;
}

int batch_enqueue(ddsp_batch &B, float thr, cudaStream_t s) {
  cudaError_t e = launch_batch_reset(B.d_queue, kMaxGroups, B.d_counts,
                                     B.nbeams, s);
  if (B.mode == DDSP_BATCH_PER_BEAM) {
    if (e == cudaSuccess) e = batch_dedisperse_per_beam(B, s);
    if (e == cudaSuccess)
      e = launch_sps_batch(B.d_sb, B.nbeams, B.sps_blocks, thr, B.sps_smem,
                           B.sps_cap, s);
    return cuda_rc(e);
  }
  for (size_t gi = 0; gi < B.groups.size() && e == cudaSuccess; ++gi) {
    const BatchGroup &G = B.groups[gi];
    e = launch_dedisperse_persistent(G.tile, G.d_wsb, G.d_items, G.nitems, 0,
                                     0, B.d_queue + gi, G.smem, B.d_err,
                                     G.grid, s);
  }
  if (e == cudaSuccess)
    e = launch_sps_batch(B.d_sb, B.nbeams, B.sps_blocks, thr, B.sps_smem,
                           B.sps_cap, s);
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
    B->sps_cap = sps_bufcap(maxlen_all, wmax_all);
    if ((e = cudaMalloc(&B->d_sb, sb.size() * sizeof(SpsBeam))) != cudaSuccess ||
        (e = cudaMalloc(&B->d_counts, counts.size() * sizeof(uint32_t *))) != cudaSuccess ||
        (e = cudaMalloc(&B->d_queue, kMaxGroups * sizeof(int))) != cudaSuccess ||
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
  const int rc = batch_apply_tile(*B, t);
  if (rc == DDSP_OK && B->mode != DDSP_BATCH_PERSISTENT) {
    B->mode = DDSP_BATCH_PERSISTENT;   // a tile is a persistent-mode choice
    B->ran_direct = false;
  }
  return rc;
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
  if (grid) *grid = B->groups.empty() ? 0 : B->groups[0].grid;
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
    p.last_nwin = nwin;
    const int rc = mark_searched(p, s);
    if (rc != DDSP_OK) return rc;
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
      // every kAutotuneStride-th item of each group's cost-ordered work
      // list: the same share of every beam's work for each candidate
      std::vector<int4> sample;
      std::vector<size_t> off(B->groups.size() + 1, 0);
      size_t all = 0;
      for (size_t gi = 0; gi < B->groups.size(); ++gi) {
        const auto &items = B->groups[gi].items;
        for (size_t k = 0; k < items.size(); k += kAutotuneStride)
          sample.push_back(items[k]);
        off[gi + 1] = sample.size();
        all += items.size();
      }
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
      float best_rep = 1e30f;
      for (int r = 0; r <= reps && e == cudaSuccess; ++r) {
        launch_batch_reset(B->d_queue, kMaxGroups, B->d_counts, B->nbeams, s);
        cudaEventRecord(e0, s);
        for (size_t gi = 0; gi < B->groups.size() && e == cudaSuccess; ++gi) {
          const BatchGroup &G = B->groups[gi];
          const int n = (int)(off[gi + 1] - off[gi]);
          if (n == 0) continue;
          e = launch_dedisperse_persistent(G.tile, G.d_wsb, d_sample + off[gi],
                                           n, 0, 0, B->d_queue + gi, G.smem,
                                           B->d_err, std::min(G.grid, n), s);
        }
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float t = 0;
        cudaEventElapsedTime(&t, e0, e1);
        if (r > 0) best_rep = std::min(best_rep, t);  // first run warms up
      }
      if (e == cudaSuccess && !sample.empty())
        ms = best_rep * (float)all / (float)sample.size();
      if (ms > 0 && ms < bestms) {
        bestms = ms;
        besti = i;
      }
    }
    if (ms_out && i < cap) ms_out[i] = ms;
    ++tried;
  }
  cudaFree(d_sample);
  int rc = besti < 0 ? DDSP_E_INVALID_ARG
                     : batch_apply_tile(*B, kBatchTiles[besti]);
  B->mode = DDSP_BATCH_PERSISTENT;
  // the per-beam interleaved mode: one whole dedispersion pass per rep
  float ms_il = -1.0f;
  if (rc == DDSP_OK && batch_setup_il(*B) == DDSP_OK) {
    float best_rep = 1e30f;
    cudaError_t e = cudaSuccess;
    for (int r = 0; r <= reps && e == cudaSuccess; ++r) {
      cudaEventRecord(e0, s);
      e = batch_dedisperse_per_beam(*B, s);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float t = 0;
      cudaEventElapsedTime(&t, e0, e1);
      if (r > 0) best_rep = std::min(best_rep, t);  // first run warms up
    }
    if (e == cudaSuccess) ms_il = best_rep;
    if (ms_il > 0 && ms_il < bestms) {
      B->mode = DDSP_BATCH_PER_BEAM;
      besti = kNumBatchTiles;
    }
  }
  if (ms_out && kNumBatchTiles < cap) ms_out[kNumBatchTiles] = ms_il;
  ++tried;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (ntried) *ntried = tried;
  if (best) *best = besti;
  B->ran_direct = false;
  batch_free_graph(*B);
  return rc;
}

int ddsp_batch_set_mode(ddsp_batch *B, int mode) {
  if (!B || (mode != DDSP_BATCH_PERSISTENT && mode != DDSP_BATCH_PER_BEAM))
    return DDSP_E_INVALID_ARG;
  DeviceGuard g(B->device);
  if (mode == DDSP_BATCH_PER_BEAM) {
    cudaDeviceSynchronize();
    const int rc = batch_setup_il(*B);
    if (rc != DDSP_OK) return rc;
  }
  if (mode != B->mode) {
    batch_free_graph(*B);
    B->ran_direct = false;
    B->mode = mode;
  }
  return DDSP_OK;
}

int ddsp_batch_get_mode(const ddsp_batch *B, int *mode) {
  if (!B || !mode) return DDSP_E_INVALID_ARG;
  *mode = B->mode;
  return DDSP_OK;
}

int ddsp_batch_get_beam_tile(const ddsp_batch *B, int beam, int *dm_tile,
                             int *dm_per_thread, int *time_tile,
                             int *chan_chunk, int *group) {
  if (!B || beam < 0 || beam >= B->nbeams || B->groups.empty())
    return DDSP_E_INVALID_ARG;
  const int gi = B->group_of[beam];
  const DedispTile &t = B->groups[gi].tile;
  if (dm_tile) *dm_tile = t.dm_tile();
  if (dm_per_thread) *dm_per_thread = t.rd;
  if (time_tile) *time_tile = dedisp_time_tile(t, 8);
  if (chan_chunk) *chan_chunk = B->cc[beam];
  if (group) *group = gi;
  return DDSP_OK;
}

}  // extern "C"
