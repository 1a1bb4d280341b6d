// k_batch.cu -- many beams of uneven shape dedispersed in one persistent
// launch (the batched form of Sec.3.2), plus the small kernels that start a
// batch step (queue and count reset) and a streaming group (the same, plus
// the boxcar carry of every beam in and out of its series slot).
//
// A grid of (SMs x resident blocks) blocks loops: one thread takes the next
// work item from a device queue (atomicAdd on a counter), the block runs it
// with ws_item.cuh (producer warps stage and relayout, consumer warps
// accumulate), and the mbarrier phases continue across items through a
// running chunk counter.  Items are (beam, DM tile, time tile) triples,
// ordered by the host so that the most expensive ones start first.  All
// beams share one tile shape (warps, DM trials per thread) and one stage
// count; each beam has its own channel chunk and buffer extents, and the
// dynamic shared memory is the largest layout over the beams.  When every
// beam has the same shape the host passes no item list: item i is beam
// i / ipb, DM tile (i % ipb) % ndt, time tile (i % ipb) / ndt (DM tiles
// innermost: concurrent blocks stage overlapping windows of one time tile,
// which L2 then serves).
#include <algorithm>

#include "ws_item.cuh"

namespace ddsp {
namespace {

template <int WT, int WD, int RD>
__global__ void __launch_bounds__(32 * (WT * WD + kWsProdWarps), 2)
dedisp_persistent_kernel(const WsBeam *__restrict__ beams,
                         const int4 *__restrict__ items, int nitems,
                         int ipb, int ndt, int *queue, int nbuf, int32_t *err,
                         long long timeout_cycles) {
  constexpr int TT = 4 * 32 * kElemPerThread * WT;
  extern __shared__ __align__(16) unsigned char smem[];
  int *s_item = reinterpret_cast<int *>(smem + 64);
  if (threadIdx.x == 0) ws_init_barriers(smem, nbuf, WT * WD);
  int jbase = 0;
  while (true) {
    if (threadIdx.x == 0) *s_item = atomicAdd(queue, 1);
    __syncthreads();
    const int it = *s_item;
    if (it >= nitems) break;
    int4 w;                             // {beam, DM tile, time tile, -}
    if (items) {
      w = items[it];
    } else {
      const int r = it % ipb;
      w = make_int4(it / ipb, r % ndt, r / ndt, 0);
    }
    const WsBeam a = beams[w.x];
    const bool ok = ws_item<WT, WD, RD, uint8_t>(
        a, w.y, (int64_t)w.z * TT, jbase, smem, nbuf, err, timeout_cycles);
    jbase += (a.nchan + a.cc - 1) / a.cc;
    // every role is done with the item before the next one starts; a block
    // whose item failed stops taking work
    if (__syncthreads_or(!ok)) break;
  }
}

__global__ void batch_reset_kernel(int *queue, int nqueues,
                                   uint32_t *const *counts, int ncounts) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nqueues) queue[i] = 0;
  if (i < ncounts) *counts[i] = 0;
}

// Streaming group carry.  in: reset the queue and each beam's candidate
// count and copy the beam's carry (the last `carry` outputs of its previous
// block) to the front of its series slot; out: copy the series' last
// `carry` samples back to the beam's carry for its next block.  Rows are n
// samples, n and carry multiples of 4, n >= 2 * carry; one int4 per thread.
__global__ void serve_carry_kernel(const SpsBeam *__restrict__ beams,
                                   int32_t *const *__restrict__ carries,
                                   int nbeams, int ndm, int64_t n, int carry,
                                   bool in, int *queue) {
  const int64_t q = carry / 4;
  const int64_t total = (int64_t)nbeams * ndm * q;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (in) {
    if (i0 == 0) *queue = 0;
    if (i0 < nbeams) *beams[i0].count = 0;
  }
  for (int64_t i = i0; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(i / ((int64_t)ndm * q));
    const int64_t rem = i - (int64_t)b * ndm * q;
    const int64_t row = rem / q, c4 = rem - row * q;
    // the search only reads the series; this kernel is its one writer
    // besides the dedispersion
    int32_t *x = const_cast<int32_t *>(beams[b].series) + row * n;
    int4 *cy = reinterpret_cast<int4 *>(carries[b] + row * carry);
    if (in)
      reinterpret_cast<int4 *>(x)[c4] = cy[c4];
    else
      cy[c4] = reinterpret_cast<const int4 *>(x + n - carry)[c4];
  }
}

template <int WT, int WD, int RD>
cudaError_t launch_persistent_t(const WsBeam *d_beams, const int4 *d_items,
                                int nitems, int ipb, int ndt, int *d_queue,
                                int nbuf,
                                size_t smem, int32_t *d_err, int grid,
                                cudaStream_t s) {
  auto kern = dedisp_persistent_kernel<WT, WD, RD>;
  cudaError_t e = smem_opt_in(kern);
  if (e != cudaSuccess) return e;
  const long long timeout = 4000000000LL;  // ~2 s of SM clock
  kern<<<grid, 32 * (WT * WD + kWsProdWarps), smem, s>>>(
      d_beams, d_items, nitems, ipb, ndt, d_queue, nbuf, d_err, timeout);
  return cudaGetLastError();
}

}  // namespace

// Blocks per SM the persistent kernel can keep resident for a tile shape.
int persistent_blocks_per_sm(const DedispTile &t, size_t smem) {
  int n = 0;
  cudaError_t e = cudaSuccess;
#define DDSP_OCC(WT_, WD_, RD_)                                                \
  if (t.wt == WT_ && t.wd == WD_ && t.rd == RD_) {                             \
    auto k = dedisp_persistent_kernel<WT_, WD_, RD_>;                          \
    e = smem_opt_in(k);                                                        \
    if (e == cudaSuccess)                                                      \
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(                       \
          &n, k, 32 * (WT_ * WD_ + kWsProdWarps), smem);                       \
  }
  DDSP_OCC(4, 2, 4) DDSP_OCC(2, 4, 4) DDSP_OCC(8, 1, 4)
  DDSP_OCC(4, 2, 8) DDSP_OCC(2, 4, 8) DDSP_OCC(8, 1, 8)
#undef DDSP_OCC
  return e == cudaSuccess ? n : 0;
}

cudaError_t launch_serve_carry(const SpsBeam *d_beams,
                               int32_t *const *d_carry, int nbeams, int ndm,
                               int64_t n, int carry, bool in, int *d_queue,
                               cudaStream_t s) {
  const int64_t total = std::max<int64_t>((int64_t)nbeams * ndm * (carry / 4),
                                          nbeams);
  const int64_t blocks = std::min<int64_t>((total + 255) / 256, 148 * 16);
  serve_carry_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(
      d_beams, d_carry, nbeams, ndm, n, carry, in, d_queue);
  return cudaGetLastError();
}

cudaError_t launch_batch_reset(int *d_queue, int nqueues,
                               uint32_t *const *d_counts, int ncounts,
                               cudaStream_t s) {
  const int n = std::max(std::max(ncounts, nqueues), 1);
  batch_reset_kernel<<<(n + 255) / 256, 256, 0, s>>>(d_queue, nqueues,
                                                     d_counts, ncounts);
  return cudaGetLastError();
}

cudaError_t launch_dedisperse_persistent(const DedispTile &t,
                                         const WsBeam *d_beams,
                                         const int4 *d_items, int nitems,
                                         int ipb, int ndt, int *d_queue,
                                         size_t smem,
                                         int32_t *d_err, int grid,
                                         cudaStream_t s) {
#define DDSP_P(WT_, WD_, RD_)                                                 \
  if (t.wt == WT_ && t.wd == WD_ && t.rd == RD_)                              \
    return launch_persistent_t<WT_, WD_, RD_>(d_beams, d_items, nitems, ipb,  \
                                              ndt, d_queue, t.nbuf, smem,     \
                                              d_err, grid, s);
  DDSP_P(4, 2, 4) DDSP_P(2, 4, 4) DDSP_P(8, 1, 4)
  DDSP_P(4, 2, 8) DDSP_P(2, 4, 8) DDSP_P(8, 1, 8)
#undef DDSP_P
  return cudaErrorInvalidValue;
}

}  // namespace ddsp
