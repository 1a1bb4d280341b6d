// internal.h -- plan layout and kernel launchers shared by the library's
// translation units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "ddsp.h"

namespace ddsp {

// Device-side error word values (plan->d_err).
enum : int32_t { kErrNone = 0, kErrTimeout = 1, kErrRange = 2 };

// Bound of every device wait, in SM clock cycles (about 2 s at 2 GHz); the
// waits a block makes for its own copies in flight before it exits always
// use it, whatever a plan sets for its hand-off waits.
constexpr long long kDefaultWaitCycles = 4000000000LL;

// Dedispersion kernel geometry: 8 warps per block, each thread owns
// rd DM trials x kElemPerThread interleaved elements.
constexpr int kThreads = 256;
constexpr int kElemPerThread = 4;

// DedispTile::flags
enum : int {
  kTileSingleElemBuffer = 1,  // one element buffer, two barriers per chunk
  kTileRegisterTotals = 4,    // int32 totals in registers, not in the output
  kTileWarpSpecialized = 8,   // producer / consumer warps (k_dedisp_ws.cu)
  kTileInterleaved = 16,      // staged from pre-interleaved rows (k_dedisp_il.cu)
  kTileWide = 32,             // with kTileInterleaved: 16 consumer warps
};

struct DedispTile {
  int wt = 0;          // warps along time (0: use the direct kernel);
                       // wt * wd = 8 consumer warps, 16 for kTileWide
  int wd = 0;          // warps along DM
  int rd = 4;          // DM trials per thread (2 or 4; 4 or 8 when warp-
                       // specialised)
  int chan_chunk = 0;  // channels staged per pipeline step
  int nbuf = 2;        // raw-window stages (bulk copies in flight + 1);
                       // element stages when interleaved
  int flags = 0;       // kTile* variant switches
  int dm_tile() const { return wd * rd; }
};

struct DedispTables {
  // per (DM tile g, channel c): window start (multiple of 16, samples
  // relative to the block's first output sample), bytes to copy, and the
  // element-byte offsets of the tile's DM trials.
  int n_dm_tiles = 0;
  int dm_tile = 0;
  int span_max = 0;           // max over (g, c) of (dhi - wbase)
  int32_t *d_desc = nullptr;  // [n_dm_tiles][nchan] {window start, bytes}
  int32_t *d_relb = nullptr;  // [n_dm_tiles][nchan][dm_tile], bytes
  int32_t *d_rowmap = nullptr;// [n_dm_tiles*dm_tile] output row (-1 = pad)
};

struct Plan {
  int device = 0;
  int nchan = 0, ndm = 0, nbits = 8, nwidths = 0;
  double f_top = 0, chan_bw = 0, tsamp = 0;
  std::vector<double> dms;
  std::vector<int> widths;
  int64_t norm_window = 0;
  size_t cand_capacity = 0;

  std::vector<int32_t> delays;  // [ndm][nchan], plan order
  int32_t max_delay = 0;
  std::vector<int> order;       // DM trials sorted by DM value

  DedispTile tile;       // wt == 0: no staged tile fits, use the direct kernel
  DedispTables tab;
  int32_t *d_delays = nullptr;  // [ndm][nchan] device copy (direct kernel)

  // channel-major workspace, and the interleaved rows staged by the
  // kTileInterleaved kernel ([nchan][cm pitch] uint32)
  void *d_cm = nullptr;
  size_t cm_bytes = 0;
  void *d_il = nullptr;
  size_t il_bytes = 0;
  int64_t staged_nout = 0;    // block staged by ddsp_stage (0: none)
  int64_t staged_pitch = 0;

  // search workspace
  int64_t *d_m2 = nullptr, *d_mad4 = nullptr;
  size_t stats_cap = 0;
  int64_t last_nwin = 0;
  ddsp_cand *d_cands = nullptr;
  uint32_t *d_count = nullptr;
  int32_t *d_err = nullptr;
  int32_t *d_widths = nullptr;
  bool searched = false;
  cudaStream_t last_stream = nullptr;
  // recorded after every search launch: reading the results waits for the
  // search, not for work queued behind it on the same stream; the reads go
  // through a plan-owned non-blocking stream (a copy on the legacy default
  // stream would wait for every blocking stream's work)
  cudaEvent_t ev_search = nullptr;
  cudaStream_t copy_stream = nullptr;

  // failure detection of the interleaved dedispersion kernel: the bound of
  // its copy/compute hand-off waits in SM cycles (0: kDefaultWaitCycles),
  // and a test switch that stops the copy-issuing warp before a chunk
  // (-1: off)
  long long wait_limit = 0;
  int withhold_chunk = -1;

  // resampling (ddsp_resample): the first bin edge of every 32-bin group,
  // tabulated on the host in FP64
  void *d_rs = nullptr;
  size_t rs_bytes = 0;
};

// ---- multi-beam descriptors (device arrays built by the batch) ---------
struct SpsBeam {             // one beam of the batched search
  const int32_t *series;     // [ndm][n]
  const int32_t *widths;
  int64_t *m2, *mad4;
  ddsp_cand *cands;
  uint32_t *count;
  int32_t *err;
  int64_t n, L, nwin, block0;
  int64_t nrep;              // candidates only for start times t < nrep
  int ndm, nw;
  uint32_t cap, pad;
};

struct WsBeam;  // ws_item.cuh

// ---- launchers (each returns a cudaError_t from the launch) ------------
cudaError_t launch_unpack(const void *d_in, int64_t nsamp_in, int nchan,
                          int nbits, void *d_out, int64_t pitch,
                          cudaStream_t s);
// Columns [0, ncols) of each row only (ncols <= pitch; a multiple of 4 for
// the uint8 tile kernel).
cudaError_t launch_unpack_cols(const void *d_in, int64_t nsamp_in, int nchan,
                               int nbits, void *d_out, int64_t pitch,
                               int64_t ncols, cudaStream_t s);

// ypitch: row pitch (elements) of the plan's interleaved rows p.d_il, used
// by the kTileInterleaved tile only (which first rebuilds them from d_cm).
cudaError_t launch_dedisperse(const Plan &p, const void *d_cm, int64_t pitch,
                              int64_t nsamp_out, int32_t *d_out,
                              cudaStream_t s, int64_t ypitch = 0);
cudaError_t launch_dedisperse_direct(const Plan &p, const void *d_cm,
                                     int64_t pitch, int64_t nsamp_out,
                                     int32_t *d_out, cudaStream_t s);
int dedisp_time_tile(const DedispTile &t, int nbits);
int dedisp_elems_per_thread(const DedispTile &t);
int dedisp_segment(const DedispTile &t);   // elements per segment S
int dedisp_copy_bytes(const DedispTile &t, int span, int nbits);
bool dedisp_tile_supported(const DedispTile &t, int nbits);

size_t dedisp_smem_bytes(const DedispTile &t, int span_max, int nbits);
void dedisp_buffer_sizes(const DedispTile &t, int span_max, int nbits,
                         int *rawmax, int *elmax);
size_t dedisp_ws_smem_bytes(int chan_chunk, int dm_tile, int rawmax,
                            int elmax, int nbuf);
cudaError_t launch_dedisperse_ws(const Plan &p, const void *d_cm,
                                 int64_t pitch, int64_t nsamp_out,
                                 int32_t *d_out, cudaStream_t s, int rawmax,
                                 int elmax, size_t smem);

// One of several same-shape row sets an interleaved launch can take
// (blockIdx.z): its interleaved rows and its output.
struct IlRows {
  const uint32_t *y;
  int32_t *out;
};
constexpr int kIlMaxRows = 16;

// What the interleaved kernels need of a plan, so that a batch can run
// them on its own tables and staging rows.
struct IlLaunch {
  DedispTile tile;
  const DedispTables *tab = nullptr;
  int nchan = 0, nbits = 8;
  int32_t *d_err = nullptr;
  void *d_il = nullptr;         // interleaved rows [nchan][ypitch] uint32
  long long wait_limit = kDefaultWaitCycles;  // hand-off waits (SM cycles)
  int withhold_chunk = -1;      // test switch: producer stops before it
};
IlLaunch il_launch_of(const Plan &p);
// Rows of d_cm to interleaved rows y (v.d_il if null).  ring > 0: the rows
// are rings of `ring` samples and logical sample b sits at (t0 + b) % ring
// (t0 and ring multiples of 4).
cudaError_t launch_interleave(const IlLaunch &v, const void *d_cm,
                              int64_t pitch, int64_t nvalid, int64_t ypitch,
                              cudaStream_t s, int64_t ring = 0, int64_t t0 = 0,
                              void *y = nullptr);
// nrows (<= kIlMaxRows) same-shape row sets in one launch (blockIdx.z),
// outputs with row pitch out_pitch.
cudaError_t launch_dedisperse_il_rows(const IlLaunch &v, int64_t ypitch,
                                      int64_t nsamp_out, int64_t out_pitch,
                                      const IlRows *rows, int nrows,
                                      cudaStream_t s);
cudaError_t launch_dedisperse_il(const IlLaunch &v, int64_t ypitch,
                                 int64_t nsamp_out, int32_t *d_out,
                                 cudaStream_t s);
cudaError_t launch_dedisperse_il(const IlLaunch &v, int64_t ypitch,
                                 int64_t nsamp_out, int32_t *d_out,
                                 cudaStream_t s, int elmax, size_t smem);
size_t dedisp_il_smem_bytes(int chan_chunk, int dm_tile, int elmax, int nst);
int dedisp_il_max_stages();
cudaError_t launch_interleave(const Plan &p, const void *d_cm, int64_t pitch,
                              int64_t nvalid, int64_t ypitch, cudaStream_t s);
// Time-major input straight to the plan's interleaved rows (uint8 with
// nchan % 16 == 0 only: unpack_interleave_fused).
bool unpack_interleave_fused(const Plan &p);
cudaError_t launch_unpack_interleave(const Plan &p, const void *d_in,
                                     int64_t nsamp_in, int64_t ypitch,
                                     cudaStream_t s);
cudaError_t launch_dedisperse_il(const Plan &p, int64_t ypitch,
                                 int64_t nsamp_out, int32_t *d_out,
                                 cudaStream_t s, int elmax, size_t smem);

cudaError_t launch_sps(const Plan &p, const int32_t *d_series,
                       int64_t nsamp_out, float threshold, bool dense,
                       int32_t *d_best_w, float *d_best_snr,
                       int32_t *d_best_sum, cudaStream_t s);

int64_t sps_max_window_samples();

// Opt kernel `func` in to the largest dynamic shared memory the device
// allows (its static shared memory deducted), once per (device, kernel).
// Every launcher of a kernel shares the setting and nothing lowers it; a
// launch still gets only the dynamic size it asks for.
cudaError_t smem_opt_in(const void *func);
template <typename F>
cudaError_t smem_opt_in(F *func) {
  return smem_opt_in(reinterpret_cast<const void *>(func));
}

int persistent_blocks_per_sm(const DedispTile &t, size_t smem);
cudaError_t launch_batch_reset(int *d_queue, int nqueues,
                               uint32_t *const *d_counts, int ncounts,
                               cudaStream_t s);
// A streaming group's carry: in (d_queue reset, each beam's candidate count
// reset, carry[b][k][0, C) -> series[b][k][0, C)) before its dedispersion,
// or out (series[b][k][n - C, n) -> carry[b][k]) after it.
cudaError_t launch_serve_carry(const SpsBeam *d_beams,
                               int32_t *const *d_carry, int nbeams, int ndm,
                               int64_t n, int carry, bool in, int *d_queue,
                               cudaStream_t s);
cudaError_t launch_dedisperse_persistent(const DedispTile &t,
                                         const WsBeam *d_beams,
                                         const int4 *d_items, int nitems,
                                         int ipb, int ndt, int *d_queue,
                                         size_t smem,
                                         int32_t *d_err, int grid,
                                         cudaStream_t s);
// Search launch layout for windows of up to maxlen samples and the widest
// boxcar wmax: the buffer capacity (samples) every block lays out its shared
// memory with, and the dynamic shared memory that takes.
int64_t sps_bufcap(int64_t maxlen, int wmax);
size_t sps_smem_bytes(int64_t maxlen, int wmax);
cudaError_t launch_sps_batch(const SpsBeam *d_beams, int nbeams,
                             int64_t total_blocks, float threshold,
                             size_t smem, int64_t bufcap, cudaStream_t s);

}  // namespace ddsp

struct ddsp_plan {
  ddsp::Plan p;
};
