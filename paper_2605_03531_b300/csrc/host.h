// host.h -- host-side helpers shared by the plan (plan.cu), the multi-beam
// batch (batch.cu) and the streaming server (server.cu).
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace ddsp {

// shared-memory budgets of the staged dedispersion: two blocks per SM, or one
constexpr size_t kSmemBudgetTwoBlocks = 113 * 1024;
constexpr size_t kSmemBudgetOneBlock = 220 * 1024;

// Makes `dev` current for the scope and restores the previous device.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev)
      cudaSetDevice(prev);
  }
};

// DDSP_OK, or DDSP_E_NOMEM / DDSP_E_CUDA with the CUDA error recorded for
// ddsp_last_error_detail.
int cuda_rc(cudaError_t e);
int64_t round_up(int64_t v, int64_t m);
// Largest delay span (samples) inside one DM tile of dt trials, from the
// 16-sample-aligned window start.
int span_for(const Plan &p, int dt);
int build_tables_for(const Plan &p, const DedispTile &tile, DedispTables &tab);
// The library's default tile for plan p (the plan's own choice).
DedispTile choose_tile(const Plan &p);

// The interleaved shape a multi-beam mode (batch per beam, server) runs a
// beam with: the first of the 16-trial wide tiles, then the 16-, 8- and
// 4-trial tiles of 8 consumer warps (narrower DM tiles for coarse DM
// grids, whose delay spans inside a tile are long) whose time tile passes
// time_ok and whose two element stages fit one block per SM with the
// largest chunk (<= 16 or 8 channels); span(dt) is the beam's delay span
// inside a DM tile of dt trials.  wt == 0 if none fits.
template <typename TimeOk, typename Span>
DedispTile fit_interleaved_tile(TimeOk time_ok, Span span) {
  const int wide = kTileInterleaved | kTileWide;
  const DedispTile cands[] = {{4, 4, 4, 16, 2, wide}, {8, 2, 8, 16, 2, wide},
                              {4, 2, 8, 8, 2, kTileInterleaved},
                              {8, 1, 8, 8, 2, kTileInterleaved},
                              {8, 1, 4, 8, 2, kTileInterleaved}};
  for (DedispTile t : cands) {
    if (!dedisp_tile_supported(t, 8) || !time_ok(dedisp_time_tile(t, 8)))
      continue;
    const int sp = span(t.dm_tile());
    for (int cc = t.chan_chunk; cc >= 1; --cc) {
      t.chan_chunk = cc;
      if (dedisp_smem_bytes(t, sp, 8) <= kSmemBudgetOneBlock) return t;
    }
  }
  return DedispTile{};
}
// The tile of ddsp_plan_set_tile's arguments (nonzero dm_tile), checked
// against the plan's shape; and the switch of a plan to a tile (drops a
// staged block, rebuilds the tables).
int tile_from_args(const Plan &p, int dm_tile, int dm_per_thread,
                   int chan_chunk, int stages, int flags, DedispTile *out);
int apply_tile(Plan &p, const DedispTile &t);
// At plan creation: the tile autotuned for this plan's shape on this GPU,
// if the cache file named by DDSP_TILE_CACHE holds one that still fits
// (tune.cu); p.tile is left as it is otherwise.
void apply_cached_tile(Plan &p);
void free_tables(DedispTables &t);
int ensure_stats(Plan &p, size_t n);
// Normalisation windows of an n-sample series; DDSP_E_SHAPE if one window
// (plus the widest boxcar) exceeds the search kernel's shared memory, unless
// allow_long (the plan search, which then takes its long mode).
int search_windows(const Plan &p, int64_t n, int64_t *nwin,
                   bool allow_long = false);
// Reads and clears the plan's device error word.
int read_err(Plan &p);
// after a search launch on s: records the plan's search event
int mark_searched(Plan &p, cudaStream_t s);
// waits for the plan's last search (its event, else its stream)
cudaError_t wait_search(Plan &p);
// device-to-host copy through the plan's copy stream, then waits for it
cudaError_t copy_to_host(Plan &p, void *dst, const void *src, size_t bytes);

}  // namespace ddsp
