// tune.cu -- autotuning of a single-beam plan's dedispersion tile (the
// Sec.3.2 kernels have several tile shapes; which is fastest depends on the
// channel count, the DM grid's delay spans and the GPU), and the cache that
// keeps each choice per (GPU, plan shape) in a small JSON file:
//
//   {"version": 1, "entries": [
//     {"key": "<gpu>/nchan=4096/nbits=8/ndm=1024/D=89989/span16=684",
//      "tile": [16, 4, 11, 2, 48], "ms": 37.812},
//     ...]}
//
// "tile" is (dm_tile, dm_per_thread, chan_chunk, stages, flags) as
// ddsp_plan_set_tile takes it.  ddsp_plan_create consults the file named by
// the environment variable DDSP_TILE_CACHE.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "host.h"

using namespace ddsp;

namespace {

struct CacheEntry {
  std::string key;
  int tile[5];
  float ms;
};

bool key_ok(const char *key) {
  if (!key || !*key || strlen(key) > 480) return false;
  for (const char *c = key; *c; ++c)
    if (*c == '"' || *c == '\\' || (unsigned char)*c < 0x20) return false;
  return true;
}

// Reads every entry of a cache file; a missing file is an empty cache,
// false only for a file that exists but does not parse.
bool read_cache(const char *path, std::vector<CacheEntry> &out) {
  out.clear();
  FILE *f = fopen(path, "rb");
  if (!f) return true;
  std::string s;
  char buf[4096];
  size_t n;
  while ((n = fread(buf, 1, sizeof(buf), f)) > 0) s.append(buf, n);
  fclose(f);
  size_t pos = 0;
  while (true) {
    size_t k = s.find("\"key\"", pos);
    if (k == std::string::npos) break;
    size_t q0 = s.find('"', s.find(':', k + 5) + 1);
    if (q0 == std::string::npos) return false;
    size_t q1 = s.find('"', q0 + 1);
    if (q1 == std::string::npos) return false;
    CacheEntry e;
    e.key = s.substr(q0 + 1, q1 - q0 - 1);
    size_t t = s.find("\"tile\"", q1);
    size_t b = t == std::string::npos ? t : s.find('[', t);
    if (b == std::string::npos) return false;
    const char *c = s.c_str() + b + 1;
    for (int i = 0; i < 5; ++i) {
      char *end = nullptr;
      const long v = strtol(c, &end, 10);
      if (end == c) return false;
      e.tile[i] = (int)v;
      c = end;
      while (*c == ' ' || *c == ',' || *c == '\n' || *c == '\t' || *c == '\r')
        ++c;
    }
    size_t m = s.find("\"ms\"", b);
    size_t colon = m == std::string::npos ? m : s.find(':', m);
    if (colon == std::string::npos) return false;
    e.ms = strtof(s.c_str() + colon + 1, nullptr);
    out.push_back(e);
    pos = colon + 1;
  }
  return true;
}

bool write_cache(const char *path, const std::vector<CacheEntry> &v) {
  const std::string tmp = std::string(path) + ".tmp";
  FILE *f = fopen(tmp.c_str(), "wb");
  if (!f) return false;
  fprintf(f, "{\"version\": 1, \"entries\": [\n");
  for (size_t i = 0; i < v.size(); ++i)
    fprintf(f, "  {\"key\": \"%s\", \"tile\": [%d, %d, %d, %d, %d], "
               "\"ms\": %.4f}%s\n",
            v[i].key.c_str(), v[i].tile[0], v[i].tile[1], v[i].tile[2],
            v[i].tile[3], v[i].tile[4], (double)v[i].ms,
            i + 1 < v.size() ? "," : "");
  fprintf(f, "]}\n");
  const bool ok = fclose(f) == 0;
  return ok && rename(tmp.c_str(), path) == 0;
}

// The key of a plan: GPU name and what decides the fastest tile.
std::string plan_key(const Plan &p) {
  cudaDeviceProp prop;
  std::string gpu = "unknown-gpu";
  if (cudaGetDeviceProperties(&prop, p.device) == cudaSuccess) gpu = prop.name;
  for (char &c : gpu)
    if (c == '"' || c == '\\' || c == '/' || (unsigned char)c < 0x20) c = '_';
  char buf[512];
  snprintf(buf, sizeof(buf), "%s/nchan=%d/nbits=%d/ndm=%d/D=%d/span16=%d",
           gpu.c_str(), p.nchan, p.nbits, p.ndm, p.max_delay, span_for(p, 16));
  return buf;
}

// The tiles the autotuner tries: (dm_tile, dm_per_thread, largest
// chan_chunk, flags); the chunk is the largest that fits.
struct TuneCand {
  int dt, rd, cc, flags;
};
const TuneCand kTuneCands[] = {
    {16, 4, 16, kTileInterleaved | kTileWide},
    {16, 8, 16, kTileInterleaved | kTileWide},
    {32, 8, 16, kTileInterleaved | kTileWide},
    {8, 4, 16, kTileInterleaved | kTileWide},
    {8, 8, 16, kTileInterleaved | kTileWide},
    {16, 8, 8, kTileInterleaved},
    {8, 8, 8, kTileInterleaved},
    {16, 4, 8, kTileInterleaved},
    {16, 8, 8, kTileWarpSpecialized},
    {8, 8, 8, kTileWarpSpecialized},
};
constexpr int kNumTuneCands = sizeof(kTuneCands) / sizeof(kTuneCands[0]);

}  // namespace

namespace ddsp {

void apply_cached_tile(Plan &p) {
  const char *path = getenv("DDSP_TILE_CACHE");
  if (!path || !*path) return;
  std::vector<CacheEntry> v;
  if (!read_cache(path, v)) return;
  const std::string key = plan_key(p);
  for (const CacheEntry &e : v) {
    if (e.key != key) continue;
    DedispTile t;
    if (tile_from_args(p, e.tile[0], e.tile[1], e.tile[2], e.tile[3],
                       e.tile[4], &t) == DDSP_OK)
      p.tile = t;
    return;
  }
}

}  // namespace ddsp

extern "C" {

int ddsp_tile_cache_get(const char *path, const char *key, int *tile,
                        float *ms) {
  if (!path || !key_ok(key) || !tile) return DDSP_E_INVALID_ARG;
  std::vector<CacheEntry> v;
  if (!read_cache(path, v)) return DDSP_E_INVALID_ARG;
  for (const CacheEntry &e : v) {
    if (e.key != key) continue;
    memcpy(tile, e.tile, sizeof(e.tile));
    if (ms) *ms = e.ms;
    return DDSP_OK;
  }
  return DDSP_E_STATE;
}

int ddsp_tile_cache_put(const char *path, const char *key, const int *tile,
                        float ms) {
  if (!path || !key_ok(key) || !tile) return DDSP_E_INVALID_ARG;
  std::vector<CacheEntry> v;
  if (!read_cache(path, v)) return DDSP_E_INVALID_ARG;
  CacheEntry e;
  e.key = key;
  memcpy(e.tile, tile, sizeof(e.tile));
  e.ms = ms;
  auto it = std::find_if(v.begin(), v.end(),
                         [&](const CacheEntry &x) { return x.key == e.key; });
  if (it != v.end()) *it = e;
  else v.push_back(e);
  return write_cache(path, v) ? DDSP_OK : DDSP_E_INVALID_ARG;
}

int ddsp_plan_tile_key(const ddsp_plan *h, char *buf, size_t cap) {
  if (!h || !buf || cap == 0) return DDSP_E_INVALID_ARG;
  const std::string k = plan_key(h->p);
  if (k.size() + 1 > cap) return DDSP_E_INVALID_ARG;
  memcpy(buf, k.c_str(), k.size() + 1);
  return DDSP_OK;
}

int ddsp_plan_autotune(ddsp_plan *h, const void *d_in, int64_t nsamp_in,
                       const char *cache_path, int reps, ddsp_stream_t stream,
                       float *ms_out, int cap, int *best_out) {
  if (!h || !d_in || reps < 1 || (cap > 0 && !ms_out))
    return DDSP_E_INVALID_ARG;
  Plan &p = h->p;
  const int64_t nout = nsamp_in - p.max_delay;
  if (nout <= 0) return DDSP_E_SHAPE;
  DeviceGuard g(p.device);
  cudaStream_t s = (cudaStream_t)stream;
  int32_t *d_out = nullptr;
  cudaError_t e = cudaMalloc(&d_out, (size_t)p.ndm * nout * 4);
  if (e != cudaSuccess) return cuda_rc(e);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const DedispTile before = p.tile;
  int best = -1;
  float best_ms = 0.0f;
  DedispTile best_tile;
  int best_args[5] = {0, 0, 0, 0, 0};
  for (int i = 0; i < kNumTuneCands; ++i) {
    const TuneCand &c = kTuneCands[i];
    float ms = -1.0f;
    DedispTile t;
    int cc = c.cc;
    while (cc >= 1 &&
           tile_from_args(p, c.dt, c.rd, cc, 2, c.flags, &t) != DDSP_OK)
      --cc;
    if (cc >= 1 && apply_tile(p, t) == DDSP_OK) {
      // one untimed pass (workspaces for this tile), then the best of reps
      int rc = ddsp_stage(h, d_in, nsamp_in, stream);
      if (rc == DDSP_OK) rc = ddsp_dedisperse_staged(h, nout, d_out, stream);
      for (int r = 0; r < reps && rc == DDSP_OK; ++r) {
        cudaEventRecord(e0, s);
        rc = ddsp_stage(h, d_in, nsamp_in, stream);
        if (rc == DDSP_OK) rc = ddsp_dedisperse_staged(h, nout, d_out, stream);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = DDSP_E_CUDA;
        float t_ms = 0.0f;
        cudaEventElapsedTime(&t_ms, e0, e1);
        if (rc == DDSP_OK && (ms < 0.0f || t_ms < ms)) ms = t_ms;
      }
      if (rc == DDSP_OK && read_err(p) != DDSP_OK) rc = DDSP_E_TIMEOUT;
      if (rc != DDSP_OK) ms = -1.0f;
    }
    if (i < cap) ms_out[i] = ms;
    if (ms >= 0.0f && (best < 0 || ms < best_ms)) {
      best = i;
      best_ms = ms;
      best_tile = t;
      const int a[5] = {c.dt, c.rd, cc, 2, c.flags};
      memcpy(best_args, a, sizeof(a));
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d_out);
  int rc = apply_tile(p, best >= 0 ? best_tile : before);
  if (best_out) *best_out = best;
  if (rc != DDSP_OK) return rc;
  if (best < 0) return DDSP_E_INVALID_ARG;
  if (cache_path) rc = ddsp_tile_cache_put(cache_path, plan_key(p).c_str(),
                                           best_args, best_ms);
  return rc;
}

}  // extern "C"
