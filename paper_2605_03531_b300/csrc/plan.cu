// plan.cu -- the C ABI (include/ddsp.h): argument checking, the FP64 delay
// table of Ch.1 Eq.1, tile choice and per-tile staging tables, workspace
// management, and the host ends of every call.  No compute happens here:
// every step of the path runs in the kernels of k_unpack.cu, k_dedisp.cu and
// k_sps.cu.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <set>
#include <utility>
#include <new>
#include <numeric>
#include <vector>

#include "host.h"

using namespace ddsp;

namespace ddsp {

#ifdef DDSP_BOUNDS_CHECK
// First bounds violation of any kernel of the checked build (0: none).
__device__ unsigned long long g_bounds_first = 0ull;
#endif

constexpr double kDispersionConst = 4148.808;  // s MHz^2 per (pc cm^-3)

thread_local char g_detail[256] = "";

cudaError_t smem_opt_in(const void *func) {
  static std::mutex mu;
  static std::set<std::pair<int, const void *>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({dev, func})) return cudaSuccess;
  int optin = 0;
  cudaFuncAttributes fa;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                  dev)) != cudaSuccess ||
      (e = cudaFuncGetAttributes(&fa, func)) != cudaSuccess)
    return e;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           optin - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess) done.insert({dev, func});
  return e;
}

int cuda_rc(cudaError_t e) {
  if (e == cudaSuccess) return DDSP_OK;
  snprintf(g_detail, sizeof(g_detail), "%s: %s", cudaGetErrorName(e),
           cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return DDSP_E_NOMEM;
  return DDSP_E_CUDA;
}

// Ch.1 Eq.1 with f_c = f_top + c*chan_bw and f_ref = the highest channel
// frequency; rounded to the nearest sample, ties away from zero (llround).
bool build_delays(Plan &p) {
  const double f_last = p.f_top + (double)(p.nchan - 1) * p.chan_bw;
  const double fr = p.f_top > f_last ? p.f_top : f_last;
  p.delays.resize((size_t)p.ndm * p.nchan);
  int32_t dmax = 0;
  for (int k = 0; k < p.ndm; ++k) {
    for (int c = 0; c < p.nchan; ++c) {
      const double f = p.f_top + c * p.chan_bw;
      const double x = kDispersionConst * p.dms[k] *
                       (1.0 / (f * f) - 1.0 / (fr * fr)) / p.tsamp;
      if (!(x < 2.0e9)) return false;
      const int32_t d = (int32_t)llround(x);
      p.delays[(size_t)k * p.nchan + c] = d;
      dmax = std::max(dmax, d);
    }
  }
  p.max_delay = dmax;
  return true;
}

// Largest (dhi - wbase) over all (DM tile, channel) for tiles of `dt` trials
// taken from the DM-sorted order.
int span_for(const Plan &p, int dt) {
  int span = 0;
  const int ntiles = (p.ndm + dt - 1) / dt;
  for (int g = 0; g < ntiles; ++g) {
    const int a = g * dt, b = std::min(p.ndm, a + dt) - 1;
    const int32_t *dlo = &p.delays[(size_t)p.order[a] * p.nchan];
    const int32_t *dhi = &p.delays[(size_t)p.order[b] * p.nchan];
    for (int c = 0; c < p.nchan; ++c) {
      const int wb = dlo[c] & ~15;
      span = std::max(span, dhi[c] - wb);
    }
  }
  return span;
}

void free_tables(DedispTables &t) {
  cudaFree(t.d_desc);
  cudaFree(t.d_relb);
  cudaFree(t.d_rowmap);
  t.d_desc = t.d_relb = t.d_rowmap = nullptr;
}

// Build and upload the staging tables for tile shape p.tile.
// Staging tables of plan p for tile shape `tile` into `tab` (replacing what
// it held).
int build_tables_for(const Plan &p, const DedispTile &tile, DedispTables &tab) {
  free_tables(tab);
  if (tile.wt == 0) return DDSP_OK;  // direct kernel needs none
  const int dt = tile.dm_tile();
  const int ntiles = (p.ndm + dt - 1) / dt;
  std::vector<int32_t> desc((size_t)ntiles * p.nchan * 2);
  std::vector<int32_t> relb((size_t)ntiles * p.nchan * dt);
  std::vector<int32_t> rowmap((size_t)ntiles * dt, -1);
  int span_max = 0;
  for (int g = 0; g < ntiles; ++g) {
    const int a = g * dt, nvalid = std::min(dt, p.ndm - a);
    for (int r = 0; r < dt; ++r)
      rowmap[(size_t)g * dt + r] = r < nvalid ? p.order[a + r] : -1;
    for (int c = 0; c < p.nchan; ++c) {
      // delays are non-decreasing along the DM-sorted order
      const int32_t dlo = p.delays[(size_t)p.order[a] * p.nchan + c];
      const int32_t wb = dlo & ~15;
      int span = 0;
      for (int r = 0; r < dt; ++r) {
        const int k = p.order[a + std::min(r, nvalid - 1)];
        const int32_t d = p.delays[(size_t)k * p.nchan + c];
        relb[((size_t)g * p.nchan + c) * dt + r] = 4 * (d - wb);
        span = std::max(span, d - wb);
      }
      span_max = std::max(span_max, span);
      desc[((size_t)g * p.nchan + c) * 2] = wb;
      desc[((size_t)g * p.nchan + c) * 2 + 1] =
          dedisp_copy_bytes(tile, span, p.nbits);
    }
  }
  tab.n_dm_tiles = ntiles;
  tab.dm_tile = dt;
  tab.span_max = span_max;
  cudaError_t e;
  if ((e = cudaMalloc(&tab.d_desc, desc.size() * 4)) != cudaSuccess ||
      (e = cudaMalloc(&tab.d_relb, relb.size() * 4)) != cudaSuccess ||
      (e = cudaMalloc(&tab.d_rowmap, rowmap.size() * 4)) != cudaSuccess) {
    free_tables(tab);
    return cuda_rc(e);
  }
  cudaMemcpy(tab.d_desc, desc.data(), desc.size() * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(tab.d_relb, relb.data(), relb.size() * 4, cudaMemcpyHostToDevice);
  e = cudaMemcpy(tab.d_rowmap, rowmap.data(), rowmap.size() * 4,
                 cudaMemcpyHostToDevice);
  return cuda_rc(e);
}

int build_tables(Plan &p) { return build_tables_for(p, p.tile, p.tab); }

// Default tile: the first shape (in order of preference) whose staged
// windows fit: the wide interleaved tile (one block per SM), then the
// others with two resident blocks per SM, else one block per SM, else the
// direct kernel.
DedispTile choose_tile(const Plan &p) {
  // {wt, wd, rd, cc, flags}: the interleaved kernel first (fastest on the
  // 4096-channel 1024-DM block: wide 41 ms, 8 consumer warps 48 ms, the
  // warp-specialised relayout kernel 54 ms; cc is an upper limit, the
  // largest chunk that fits is taken), then the relayout kernels, then the
  // block-synchronous kernel, then smaller staging footprints
  struct Cand { int wt, wd, rd, cc, flags; };
  constexpr int kIlWide = kTileInterleaved | kTileWide;
  const Cand prefs[] = {
      {4, 4, 4, 16, kIlWide}, {8, 2, 8, 16, kIlWide}, {16, 1, 8, 16, kIlWide},
      {8, 2, 4, 16, kIlWide},
      {4, 2, 8, 8, kTileInterleaved}, {8, 1, 8, 8, kTileInterleaved},
      {4, 2, 4, 8, kTileInterleaved},
      {4, 2, 8, 8, kTileWarpSpecialized}, {8, 1, 8, 8, kTileWarpSpecialized},
      {4, 2, 4, 8, kTileSingleElemBuffer | kTileRegisterTotals},
      {4, 2, 4, 6, kTileSingleElemBuffer}, {8, 1, 4, 4, kTileSingleElemBuffer},
      {8, 1, 4, 2, kTileSingleElemBuffer}, {8, 1, 2, 2, kTileSingleElemBuffer},
      {8, 1, 2, 1, kTileSingleElemBuffer}};
  // the wide tiles (one block per SM) against the one-block budget first,
  // then the rest with two blocks per SM, then with one
  for (int pass = 0; pass < 3; ++pass) {
    const size_t budget = pass == 1 ? kSmemBudgetTwoBlocks : kSmemBudgetOneBlock;
    for (const Cand &c : prefs) {
      if (((c.flags & kTileWide) != 0) != (pass == 0)) continue;
      DedispTile t;
      t.wt = c.wt;
      t.wd = c.wd;
      t.rd = c.rd;
      t.chan_chunk = c.cc;
      t.flags = c.flags;
      if (!dedisp_tile_supported(t, p.nbits)) continue;
      const int span = span_for(p, t.dm_tile());
      if (c.flags & kTileInterleaved) {
        // two element stages of the largest chunk that fits: each chunk
        // costs the consumers a fixed synchronisation latency, which larger
        // chunks amortise better than a deeper ring hides it (4096-channel
        // 1024-DM block, 8 consumer warps: 7 channels x 2 stages 49 ms, 4 x
        // 3 54 ms, 2 x 6 64 ms; wide: 11 x 2 42 ms, 7 x 3 43 ms)
        t.nbuf = 2;
        for (int cc = c.cc; cc >= 2; --cc) {
          t.chan_chunk = cc;
          if (dedisp_smem_bytes(t, span, p.nbits) <= budget) return t;
        }
        continue;
      }
      if (c.flags & kTileWarpSpecialized) {
        t.nbuf = 2;
        for (int cc = c.cc; cc >= 2; --cc) {
          t.chan_chunk = cc;
          if (dedisp_smem_bytes(t, span, p.nbits) <= budget) return t;
        }
        continue;
      }
      for (int nbuf : {3, 2}) {
        t.nbuf = nbuf;
        if (dedisp_smem_bytes(t, span, p.nbits) <= budget) return t;
      }
    }
  }
  return DedispTile{};  // direct kernel
}

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

int64_t cm_pitch(const Plan &p, int64_t nsamp_out) {
  int64_t span_out;
  if (p.tile.wt > 0) {
    const int tt = dedisp_time_tile(p.tile, p.nbits);
    span_out = round_up(nsamp_out, tt);
  } else {
    span_out = nsamp_out;
  }
  return round_up(span_out + p.max_delay + 64, 128);
}

int ensure_cm(Plan &p, size_t bytes) {
  if (bytes <= p.cm_bytes) return DDSP_OK;
  cudaDeviceSynchronize();
  cudaFree(p.d_cm);
  p.d_cm = nullptr;
  p.cm_bytes = 0;
  cudaError_t e = cudaMalloc(&p.d_cm, bytes);
  if (e != cudaSuccess) return cuda_rc(e);
  p.cm_bytes = bytes;
  return DDSP_OK;
}

// Interleaved rows for the kTileInterleaved tile: [nchan][pitch] uint32.
int ensure_il(Plan &p, int64_t pitch) {
  if (!(p.tile.flags & kTileInterleaved)) return DDSP_OK;
  const size_t bytes = (size_t)p.nchan * pitch * 4;
  if (bytes <= p.il_bytes) return DDSP_OK;
  cudaDeviceSynchronize();
  cudaFree(p.d_il);
  p.d_il = nullptr;
  p.il_bytes = 0;
  cudaError_t e = cudaMalloc(&p.d_il, bytes);
  if (e != cudaSuccess) return cuda_rc(e);
  p.il_bytes = bytes;
  return DDSP_OK;
}

int ensure_stats(Plan &p, size_t n) {
  if (n <= p.stats_cap) return DDSP_OK;
  cudaDeviceSynchronize();
  cudaFree(p.d_m2);
  cudaFree(p.d_mad4);
  p.d_m2 = p.d_mad4 = nullptr;
  p.stats_cap = 0;
  cudaError_t e;
  if ((e = cudaMalloc(&p.d_m2, n * 8)) != cudaSuccess ||
      (e = cudaMalloc(&p.d_mad4, n * 8)) != cudaSuccess) {
    cudaFree(p.d_m2);
    p.d_m2 = nullptr;
    return cuda_rc(e);
  }
  p.stats_cap = n;
  return DDSP_OK;
}

void release(Plan &p) {
  free_tables(p.tab);
  cudaFree(p.d_delays);
  cudaFree(p.d_cm);
  cudaFree(p.d_il);
  cudaFree(p.d_m2);
  cudaFree(p.d_mad4);
  cudaFree(p.d_cands);
  cudaFree(p.d_count);
  cudaFree(p.d_err);
  cudaFree(p.d_widths);
  cudaFree(p.d_rs);
  if (p.ev_search) cudaEventDestroy(p.ev_search);
  if (p.copy_stream) cudaStreamDestroy(p.copy_stream);
  p.ev_search = nullptr;
  p.copy_stream = nullptr;
}

int mark_searched(Plan &p, cudaStream_t s) {
  p.searched = true;
  p.last_stream = s;
  cudaError_t e = cudaSuccess;
  if (!p.ev_search)
    e = cudaEventCreateWithFlags(&p.ev_search, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(p.ev_search, s);
  return cuda_rc(e);
}

cudaError_t wait_search(Plan &p) {
  return p.ev_search ? cudaEventSynchronize(p.ev_search)
                     : cudaStreamSynchronize(p.last_stream);
}

cudaError_t copy_to_host(Plan &p, void *dst, const void *src, size_t bytes) {
  cudaError_t e = cudaSuccess;
  if (!p.copy_stream)
    e = cudaStreamCreateWithFlags(&p.copy_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, p.copy_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p.copy_stream);
  return e;
}

int search_windows(const Plan &p, int64_t n, int64_t *nwin, bool allow_long) {
  const int64_t L = p.norm_window;
  *nwin = (L <= 0) ? 1 : std::max<int64_t>(1, n / L);
  const int64_t maxlen =
      (L <= 0 || *nwin == 1) ? n : std::max(L, n - (*nwin - 1) * L);
  if (!allow_long && maxlen + p.widths.back() > sps_max_window_samples())
    return DDSP_E_SHAPE;
  if (*nwin > 0x7fffffff) return DDSP_E_SHAPE;
  return DDSP_OK;
}

int read_err(Plan &p) {
  int32_t e = 0;
  if (copy_to_host(p, &e, p.d_err, 4) != cudaSuccess) return DDSP_E_CUDA;
  if (e != kErrNone) {
    cudaMemsetAsync(p.d_err, 0, 4, p.copy_stream);
    cudaStreamSynchronize(p.copy_stream);
  }
  if (e == kErrTimeout) return DDSP_E_TIMEOUT;
  if (e == kErrRange) return DDSP_E_RANGE;
  return DDSP_OK;
}

}  // namespace ddsp

extern "C" {

const char *ddsp_last_error_detail(void) { return g_detail; }

const char *ddsp_error_string(int code) {
  switch (code) {
    case DDSP_OK: return "ok";
    case DDSP_E_INVALID_ARG: return "invalid argument";
    case DDSP_E_SHAPE: return "input shape does not fit the plan";
    case DDSP_E_CUDA: return "CUDA runtime error";
    case DDSP_E_NOMEM: return "out of memory";
    case DDSP_E_TIMEOUT: return "bounded device wait expired";
    case DDSP_E_TRUNCATED: return "more candidates than capacity";
    case DDSP_E_RANGE: return "series window range too large";
    case DDSP_E_STATE: return "call out of order";
    default: return "unknown error";
  }
}

static int check_band(int nchan, double f_top_mhz, double chan_bw_mhz,
                      double tsamp_s, const double *dm_list, int ndm) {
  if (nchan <= 0 || ndm <= 0 || !dm_list) return DDSP_E_INVALID_ARG;
  if (!(f_top_mhz > 0) || !isfinite(f_top_mhz) || chan_bw_mhz == 0 ||
      !isfinite(chan_bw_mhz) || !(tsamp_s > 0) || !isfinite(tsamp_s))
    return DDSP_E_INVALID_ARG;
  const double f_last = f_top_mhz + (double)(nchan - 1) * chan_bw_mhz;
  if (!(f_last > 0)) return DDSP_E_INVALID_ARG;
  for (int k = 0; k < ndm; ++k)
    if (!(dm_list[k] >= 0) || !isfinite(dm_list[k])) return DDSP_E_INVALID_ARG;
  return DDSP_OK;
}

int ddsp_delay_table(int nchan, double f_top_mhz, double chan_bw_mhz,
                     double tsamp_s, const double *dm_list, int ndm,
                     int32_t *host_out, int32_t *max_delay) {
  int rc = check_band(nchan, f_top_mhz, chan_bw_mhz, tsamp_s, dm_list, ndm);
  if (rc != DDSP_OK || !host_out) return DDSP_E_INVALID_ARG;
  Plan p;
  p.nchan = nchan;
  p.ndm = ndm;
  p.f_top = f_top_mhz;
  p.chan_bw = chan_bw_mhz;
  p.tsamp = tsamp_s;
  p.dms.assign(dm_list, dm_list + ndm);
  if (!build_delays(p)) return DDSP_E_INVALID_ARG;
  memcpy(host_out, p.delays.data(), p.delays.size() * 4);
  if (max_delay) *max_delay = p.max_delay;
  return DDSP_OK;
}

int ddsp_plan_create(ddsp_plan **out, int nchan, double f_top_mhz,
                     double chan_bw_mhz, double tsamp_s, const double *dm_list,
                     int ndm, const int *widths, int nwidths, int nbits,
                     int64_t norm_window, size_t cand_capacity) {
  if (!out) return DDSP_E_INVALID_ARG;
  *out = nullptr;
  if (ndm > 65535 || !widths || nwidths <= 0 || nwidths > 11 ||
      (nbits != 8 && nbits != 16) || norm_window < 0 || cand_capacity == 0 ||
      cand_capacity > 0xffffffffu)
    return DDSP_E_INVALID_ARG;
  if (check_band(nchan, f_top_mhz, chan_bw_mhz, tsamp_s, dm_list, ndm) !=
      DDSP_OK)
    return DDSP_E_INVALID_ARG;
  for (int i = 0; i < nwidths; ++i) {
    const int w = widths[i];
    if (w < 1 || w > 1024 || (w & (w - 1)) != 0) return DDSP_E_INVALID_ARG;
    if (i > 0 && w <= widths[i - 1]) return DDSP_E_INVALID_ARG;
  }

  ddsp_plan *h = new (std::nothrow) ddsp_plan;
  if (!h) return DDSP_E_NOMEM;
  Plan &p = h->p;
  cudaGetDevice(&p.device);
  p.nchan = nchan;
  p.ndm = ndm;
  p.nbits = nbits;
  p.nwidths = nwidths;
  p.f_top = f_top_mhz;
  p.chan_bw = chan_bw_mhz;
  p.tsamp = tsamp_s;
  p.dms.assign(dm_list, dm_list + ndm);
  p.widths.assign(widths, widths + nwidths);
  p.norm_window = norm_window;
  p.cand_capacity = cand_capacity;
  if (!build_delays(p)) {
    delete h;
    return DDSP_E_INVALID_ARG;
  }
  p.order.resize(ndm);
  std::iota(p.order.begin(), p.order.end(), 0);
  std::stable_sort(p.order.begin(), p.order.end(),
                   [&](int a, int b) { return p.dms[a] < p.dms[b]; });
  p.tile = choose_tile(p);
  apply_cached_tile(p);   // a tile autotuned for this shape, if cached

  int rc = build_tables(p);
  cudaError_t e = cudaSuccess;
  if (rc == DDSP_OK) {
    if ((e = cudaMalloc(&p.d_delays, p.delays.size() * 4)) != cudaSuccess ||
        (e = cudaMalloc(&p.d_cands, cand_capacity * sizeof(ddsp_cand))) !=
            cudaSuccess ||
        (e = cudaMalloc(&p.d_count, 4)) != cudaSuccess ||
        (e = cudaMalloc(&p.d_err, 4)) != cudaSuccess ||
        (e = cudaMalloc(&p.d_widths, 4 * nwidths)) != cudaSuccess)
      rc = cuda_rc(e);
  }
  if (rc == DDSP_OK) {
    cudaMemcpy(p.d_delays, p.delays.data(), p.delays.size() * 4,
               cudaMemcpyHostToDevice);
    cudaMemcpy(p.d_widths, p.widths.data(), 4 * nwidths, cudaMemcpyHostToDevice);
    cudaMemset(p.d_count, 0, 4);
    e = cudaMemset(p.d_err, 0, 4);
    rc = cuda_rc(e);
  }
  if (rc != DDSP_OK) {
    release(p);
    delete h;
    return rc;
  }
  *out = h;
  return DDSP_OK;
}

void ddsp_plan_destroy(ddsp_plan *h) {
  if (!h) return;
  DeviceGuard g(h->p.device);
  cudaDeviceSynchronize();
  release(h->p);
  delete h;
}

int ddsp_plan_nsamp_out(const ddsp_plan *h, int64_t nsamp_in, int64_t *nsamp_out) {
  if (!h || !nsamp_out) return DDSP_E_INVALID_ARG;
  const int64_t n = nsamp_in - h->p.max_delay;
  if (n <= 0) return DDSP_E_SHAPE;
  *nsamp_out = n;
  return DDSP_OK;
}

int ddsp_plan_max_delay(const ddsp_plan *h, int32_t *D) {
  if (!h || !D) return DDSP_E_INVALID_ARG;
  *D = h->p.max_delay;
  return DDSP_OK;
}

int ddsp_plan_get_delays(const ddsp_plan *h, int32_t *host_out) {
  if (!h || !host_out) return DDSP_E_INVALID_ARG;
  memcpy(host_out, h->p.delays.data(), h->p.delays.size() * 4);
  return DDSP_OK;
}

int ddsp_plan_set_tile(ddsp_plan *h, int dm_tile, int dm_per_thread,
                       int chan_chunk, int stages, int flags) {
  if (!h) return DDSP_E_INVALID_ARG;
  Plan &p = h->p;
  DeviceGuard g(p.device);
  DedispTile t;
  if (dm_tile == 0) {
    t = choose_tile(p);
  } else if (dm_tile == -1) {
    t = DedispTile{};  // direct kernel
  } else {
    const int rc = tile_from_args(p, dm_tile, dm_per_thread, chan_chunk,
                                  stages, flags, &t);
    if (rc != DDSP_OK) return rc;
  }
  return apply_tile(p, t);
}

}  // extern "C"

namespace ddsp {

int tile_from_args(const Plan &p, int dm_tile, int dm_per_thread,
                   int chan_chunk, int stages, int flags, DedispTile *out) {
  DedispTile t;
  t.rd = dm_per_thread;
  if (t.rd != 2 && t.rd != 4 && t.rd != 8) return DDSP_E_INVALID_ARG;
  if (dm_tile <= 0 || dm_tile % t.rd) return DDSP_E_INVALID_ARG;
  t.wd = dm_tile / t.rd;
  if (t.wd <= 0 || (kThreads / 32) % t.wd) return DDSP_E_INVALID_ARG;
  t.wt = (kThreads / 32) / t.wd * ((flags & kTileWide) ? 2 : 1);
  t.chan_chunk = chan_chunk;
  t.nbuf = stages;
  if (flags & ~(kTileSingleElemBuffer | kTileRegisterTotals |
                kTileWarpSpecialized | kTileInterleaved | kTileWide))
    return DDSP_E_INVALID_ARG;
  t.flags = flags;
  if (!dedisp_tile_supported(t, p.nbits)) return DDSP_E_INVALID_ARG;
  const int span = span_for(p, t.dm_tile());
  if (dedisp_smem_bytes(t, span, p.nbits) > kSmemBudgetOneBlock)
    return DDSP_E_INVALID_ARG;
  *out = t;
  return DDSP_OK;
}

int apply_tile(Plan &p, const DedispTile &t) {
  cudaDeviceSynchronize();
  p.tile = t;
  p.staged_nout = 0;   // a staged block belongs to the tile that staged it
  if (!(t.flags & kTileInterleaved)) {
    cudaFree(p.d_il);
    p.d_il = nullptr;
    p.il_bytes = 0;
  }
  return build_tables(p);
}

}  // namespace ddsp

extern "C" {

int ddsp_bounds_check_status(int *enabled, uint64_t *first) {
  if (!enabled || !first) return DDSP_E_INVALID_ARG;
#ifdef DDSP_BOUNDS_CHECK
  *enabled = 1;
  unsigned long long v = 0, zero = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess)
    e = cudaMemcpyFromSymbol(&v, g_bounds_first, sizeof(v));
  if (e == cudaSuccess && v)
    e = cudaMemcpyToSymbol(g_bounds_first, &zero, sizeof(zero));
  if (e != cudaSuccess) return cuda_rc(e);
  *first = v;
#else
  *enabled = 0;
  *first = 0;
#endif
  return DDSP_OK;
}

int ddsp_plan_set_wait_limit(ddsp_plan *h, int64_t cycles) {
  if (!h || cycles < 0) return DDSP_E_INVALID_ARG;
  h->p.wait_limit = cycles;
  return DDSP_OK;
}

int ddsp_plan_withhold_copy(ddsp_plan *h, int chunk) {
  if (!h || chunk < -1) return DDSP_E_INVALID_ARG;
  h->p.withhold_chunk = chunk;
  return DDSP_OK;
}

int ddsp_plan_get_tile(const ddsp_plan *h, int *dm_tile, int *dm_per_thread,
                       int *time_tile, int *chan_chunk, int *stages,
                       int *flags) {
  if (!h) return DDSP_E_INVALID_ARG;
  const Plan &p = h->p;
  const bool staged = p.tile.wt > 0;
  if (dm_tile) *dm_tile = staged ? p.tile.dm_tile() : -1;
  if (dm_per_thread) *dm_per_thread = staged ? p.tile.rd : 0;
  if (time_tile) *time_tile = staged ? dedisp_time_tile(p.tile, p.nbits) : 0;
  if (chan_chunk) *chan_chunk = staged ? p.tile.chan_chunk : 0;
  if (stages) *stages = staged ? p.tile.nbuf : 0;
  if (flags) *flags = staged ? p.tile.flags : 0;
  return DDSP_OK;
}

int ddsp_unpack(ddsp_plan *h, const void *d_in, int64_t nsamp_in, void *d_out,
                int64_t pitch, ddsp_stream_t stream) {
  if (!h || !d_in || !d_out || nsamp_in <= 0 || pitch < nsamp_in ||
      (pitch % 128) != 0 || ((uintptr_t)d_in & 15) || ((uintptr_t)d_out & 15))
    return DDSP_E_INVALID_ARG;
  Plan &p = h->p;
  DeviceGuard g(p.device);
  return cuda_rc(launch_unpack(d_in, nsamp_in, p.nchan, p.nbits, d_out, pitch,
                               (cudaStream_t)stream));
}

// Stage a time-major block into the plan's workspace for the current tile:
// channel-major rows (unpack), plus or instead of them (uint8, nchan % 16
// == 0) the interleaved rows of the kTileInterleaved tile.
static int stage_block(Plan &p, const void *d_in, int64_t nsamp_in,
                       cudaStream_t s) {
  p.staged_nout = 0;
  const int64_t nout = nsamp_in - p.max_delay;
  if (nout <= 0) return DDSP_E_SHAPE;
  const int64_t pitch = cm_pitch(p, nout);
  const bool il = p.tile.wt > 0 && (p.tile.flags & kTileInterleaved);
  const bool fused = il && unpack_interleave_fused(p);
  int rc = il ? ensure_il(p, pitch) : DDSP_OK;
  if (rc == DDSP_OK && !fused)
    rc = ensure_cm(p, (size_t)p.nchan * pitch * (p.nbits / 8));
  if (rc != DDSP_OK) return rc;
  cudaError_t e;
  if (fused) {
    e = launch_unpack_interleave(p, d_in, nsamp_in, pitch, s);
  } else {
    e = launch_unpack(d_in, nsamp_in, p.nchan, p.nbits, p.d_cm, pitch, s);
    if (e == cudaSuccess && il)
      e = launch_interleave(p, p.d_cm, pitch, nsamp_in, pitch, s);
  }
  if (e != cudaSuccess) return cuda_rc(e);
  p.staged_nout = nout;
  p.staged_pitch = pitch;
  return DDSP_OK;
}

static int dedisperse_staged(Plan &p, int32_t *d_out, cudaStream_t s) {
  const int64_t nout = p.staged_nout, pitch = p.staged_pitch;
  cudaError_t e;
  if (p.tile.wt == 0)
    e = launch_dedisperse_direct(p, p.d_cm, pitch, nout, d_out, s);
  else if (p.tile.flags & kTileInterleaved)
    e = launch_dedisperse(p, nullptr, pitch, nout, d_out, s, pitch);
  else
    e = launch_dedisperse(p, p.d_cm, pitch, nout, d_out, s, pitch);
  return cuda_rc(e);
}

int ddsp_stage(ddsp_plan *h, const void *d_in, int64_t nsamp_in,
               ddsp_stream_t stream) {
  if (!h || !d_in || ((uintptr_t)d_in & 15)) return DDSP_E_INVALID_ARG;
  Plan &p = h->p;
  DeviceGuard g(p.device);
  return stage_block(p, d_in, nsamp_in, (cudaStream_t)stream);
}

int ddsp_dedisperse_staged(ddsp_plan *h, int64_t nsamp_out, int32_t *d_out,
                           ddsp_stream_t stream) {
  if (!h || !d_out) return DDSP_E_INVALID_ARG;
  Plan &p = h->p;
  if (p.staged_nout <= 0) return DDSP_E_STATE;
  if (nsamp_out != p.staged_nout) return DDSP_E_SHAPE;
  DeviceGuard g(p.device);
  return dedisperse_staged(p, d_out, (cudaStream_t)stream);
}

int ddsp_dedisperse(ddsp_plan *h, const void *d_in, int64_t nsamp_in,
                    int32_t *d_out, ddsp_stream_t stream) {
  if (!h || !d_in || !d_out || ((uintptr_t)d_in & 15))
    return DDSP_E_INVALID_ARG;
  Plan &p = h->p;
  DeviceGuard g(p.device);
  cudaStream_t s = (cudaStream_t)stream;
  int rc = stage_block(p, d_in, nsamp_in, s);
  if (rc != DDSP_OK) return rc;
  return dedisperse_staged(p, d_out, s);
}

int ddsp_plan_cm_pitch(const ddsp_plan *h, int64_t nsamp_out, int64_t *pitch) {
  if (!h || !pitch || nsamp_out <= 0) return DDSP_E_INVALID_ARG;
  *pitch = cm_pitch(h->p, nsamp_out);
  return DDSP_OK;
}

int ddsp_dedisperse_cm(ddsp_plan *h, const void *d_cm, int64_t pitch,
                       int64_t nsamp_out, int32_t *d_out, ddsp_stream_t stream) {
  if (!h || !d_cm || !d_out || nsamp_out <= 0 || ((uintptr_t)d_cm & 15) ||
      (pitch % 128) != 0)
    return DDSP_E_INVALID_ARG;
  Plan &p = h->p;
  const int64_t ypitch = cm_pitch(p, nsamp_out);
  if (pitch < ypitch) return DDSP_E_SHAPE;
  DeviceGuard g(p.device);
  int rc = ensure_il(p, ypitch);
  if (rc != DDSP_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e =
      p.tile.wt > 0
          ? launch_dedisperse(p, d_cm, pitch, nsamp_out, d_out, s, ypitch)
          : launch_dedisperse_direct(p, d_cm, pitch, nsamp_out, d_out, s);
  return cuda_rc(e);
}

static int run_search(ddsp_plan *h, const int32_t *d_series, int64_t n,
                      float threshold, bool dense, int32_t *bw, float *bs,
                      int32_t *bsum, ddsp_stream_t stream) {
  if (!h || !d_series || n <= 0 || n > 0x7fffffffLL) return DDSP_E_INVALID_ARG;
  if (!dense && !(threshold > 0.0f && isfinite(threshold)))
    return DDSP_E_INVALID_ARG;
  Plan &p = h->p;
  DeviceGuard g(p.device);
  int64_t nwin;
  // windows longer than the on-chip limit take the two-pass long mode
  int rc = search_windows(p, n, &nwin, true);
  if (rc != DDSP_OK) return rc;
  if (nwin > 0x7fffffff) return DDSP_E_SHAPE;
  rc = ensure_stats(p, (size_t)nwin * p.ndm);
  if (rc != DDSP_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(p.d_count, 0, 4, s);
  if (e != cudaSuccess) return cuda_rc(e);
  e = launch_sps(p, d_series, n, threshold, dense, bw, bs, bsum, s);
  if (e != cudaSuccess) return cuda_rc(e);
  p.last_nwin = nwin;
  return mark_searched(p, s);
}

int ddsp_single_pulse_search(ddsp_plan *h, const int32_t *d_series,
                             int64_t nsamp_out, float threshold,
                             ddsp_stream_t stream) {
  return run_search(h, d_series, nsamp_out, threshold, false, nullptr, nullptr,
                    nullptr, stream);
}

int ddsp_single_pulse_search_dense(ddsp_plan *h, const int32_t *d_series,
                                   int64_t nsamp_out, int32_t *d_best_w,
                                   float *d_best_snr, int32_t *d_best_sum,
                                   ddsp_stream_t stream) {
  if (!d_best_w || !d_best_snr || !d_best_sum) return DDSP_E_INVALID_ARG;
  return run_search(h, d_series, nsamp_out, 1.0f, true, d_best_w, d_best_snr,
                    d_best_sum, stream);
}

int ddsp_plan_get_stats(ddsp_plan *h, int64_t *m2, int64_t *mad4, int64_t cap,
                        int64_t *nwin) {
  if (!h || !nwin) return DDSP_E_INVALID_ARG;
  Plan &p = h->p;
  if (!p.searched) return DDSP_E_STATE;
  DeviceGuard g(p.device);
  *nwin = p.last_nwin;
  if (!m2 && !mad4) return DDSP_OK;
  const int64_t n = p.last_nwin * p.ndm;
  if (cap < n) return DDSP_E_INVALID_ARG;
  cudaError_t e = wait_search(p);
  if (e != cudaSuccess) return cuda_rc(e);
  if (m2) e = copy_to_host(p, m2, p.d_m2, n * 8);
  if (e == cudaSuccess && mad4) e = copy_to_host(p, mad4, p.d_mad4, n * 8);
  return cuda_rc(e);
}

int ddsp_candidates_fetch(ddsp_plan *h, ddsp_cand *host_buf, size_t cap,
                          size_t *n_total) {
  if (!h || !n_total || (cap > 0 && !host_buf)) return DDSP_E_INVALID_ARG;
  Plan &p = h->p;
  if (!p.searched) return DDSP_E_STATE;
  DeviceGuard g(p.device);
  cudaError_t e = wait_search(p);
  if (e != cudaSuccess) return cuda_rc(e);
  uint32_t cnt = 0;
  e = copy_to_host(p, &cnt, p.d_count, 4);
  if (e != cudaSuccess) return cuda_rc(e);
  *n_total = cnt;
  const size_t stored = std::min<size_t>(cnt, p.cand_capacity);
  const size_t ncopy = std::min(stored, cap);
  if (ncopy) {
    e = copy_to_host(p, host_buf, p.d_cands, ncopy * sizeof(ddsp_cand));
    if (e != cudaSuccess) return cuda_rc(e);
    std::sort(host_buf, host_buf + ncopy,
              [](const ddsp_cand &a, const ddsp_cand &b) {
                return a.dm_idx != b.dm_idx ? a.dm_idx < b.dm_idx : a.t < b.t;
              });
  }
  int rc = read_err(p);
  if (rc != DDSP_OK) return rc;
  return ncopy < cnt ? DDSP_E_TRUNCATED : DDSP_OK;
}

int ddsp_candidates_count(ddsp_plan *h, size_t *n_total) {
  if (!h || !n_total) return DDSP_E_INVALID_ARG;
  Plan &p = h->p;
  if (!p.searched) return DDSP_E_STATE;
  DeviceGuard g(p.device);
  cudaError_t e = wait_search(p);
  if (e != cudaSuccess) return cuda_rc(e);
  uint32_t cnt = 0;
  e = copy_to_host(p, &cnt, p.d_count, 4);
  if (e != cudaSuccess) return cuda_rc(e);
  *n_total = cnt;
  return read_err(p);
}

int ddsp_candidates_fetch_dm_range(ddsp_plan *h, uint32_t dm_lo,
                                   uint32_t dm_hi, ddsp_cand *host_buf,
                                   size_t cap, size_t *n_range,
                                   size_t *n_total) {
  if (!h || !n_range || !n_total || dm_hi < dm_lo || (cap > 0 && !host_buf))
    return DDSP_E_INVALID_ARG;
  Plan &p = h->p;
  if (!p.searched) return DDSP_E_STATE;
  DeviceGuard g(p.device);
  cudaError_t e = wait_search(p);
  if (e != cudaSuccess) return cuda_rc(e);
  uint32_t cnt = 0;
  e = copy_to_host(p, &cnt, p.d_count, 4);
  if (e != cudaSuccess) return cuda_rc(e);
  *n_total = cnt;
  const size_t stored = std::min<size_t>(cnt, p.cand_capacity);
  // stream the stored records through a bounded host buffer, keep the range
  const size_t piece = (size_t)1 << 22;
  std::vector<ddsp_cand> tmp(std::min(stored, piece));
  size_t found = 0, kept = 0;
  for (size_t off = 0; off < stored; off += piece) {
    const size_t n = std::min(piece, stored - off);
    e = copy_to_host(p, tmp.data(), p.d_cands + off, n * sizeof(ddsp_cand));
    if (e != cudaSuccess) return cuda_rc(e);
    for (size_t i = 0; i < n; ++i) {
      if (tmp[i].dm_idx >= dm_lo && tmp[i].dm_idx < dm_hi) {
        if (kept < cap) host_buf[kept++] = tmp[i];
        ++found;
      }
    }
  }
  std::sort(host_buf, host_buf + kept,
            [](const ddsp_cand &a, const ddsp_cand &b) {
              return a.dm_idx != b.dm_idx ? a.dm_idx < b.dm_idx : a.t < b.t;
            });
  *n_range = found;
  int rc = read_err(p);
  if (rc != DDSP_OK) return rc;
  return (found > kept || stored < cnt) ? DDSP_E_TRUNCATED : DDSP_OK;
}

int ddsp_plan_check(ddsp_plan *h, ddsp_stream_t stream) {
  if (!h) return DDSP_E_INVALID_ARG;
  Plan &p = h->p;
  DeviceGuard g(p.device);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_rc(e);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_rc(e);
  return read_err(p);
}

}  // extern "C"

// ===========================================================================
// Batches: many beams (plans) of uneven shape processed by one persistent
// dedispersion launch, one batched unpack and one batched search launch,
// optionally replayed from a captured CUDA graph.
// ===========================================================================
