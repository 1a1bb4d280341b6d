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
void free_tables(DedispTables &t);
int ensure_stats(Plan &p, size_t n);
// Normalisation windows of an n-sample series; DDSP_E_SHAPE if one window
// (plus the widest boxcar) exceeds the search kernel's shared memory.
int search_windows(const Plan &p, int64_t n, int64_t *nwin);
// Reads and clears the plan's device error word.
int read_err(Plan &p);

}  // namespace ddsp
