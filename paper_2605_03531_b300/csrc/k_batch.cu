// k_batch.cu -- many beams of uneven shape dedispersed in one persistent
// launch (the batched form of Sec.3.2), plus the small reset kernel that
// starts a batch step.
//
// A grid of (SMs x resident blocks) blocks loops: one thread takes the next
// work item from a device queue (atomicAdd on a counter), the block runs it
// with ws_item.cuh (producer warps stage and relayout, consumer warps
// accumulate), and the mbarrier phases continue across items through a
// running chunk counter.  Items are (beam, DM tile, time tile) triples,
// ordered by the host so that the most expensive ones start first; all
// beams share one tile shape and one shared-memory layout (the maxima over
// the beams).
#include "ws_item.cuh"

namespace ddsp {
namespace {

template <int WT, int WD, int RD>
__global__ void __launch_bounds__(32 * (WT * WD + kWsProdWarps), 2)
dedisp_persistent_kernel(const WsBeam *__restrict__ beams,
                         const int4 *__restrict__ items, int nitems,
                         int *queue, int cc, int nbuf, int rawmax, int elmax,
                         int32_t *err, long long timeout_cycles) {
  constexpr int TT = 4 * 32 * kElemPerThread * WT;
  constexpr int DT = RD * WD;
  extern __shared__ __align__(16) unsigned char smem[];
  const WsLayout L(cc, DT, rawmax, elmax, nbuf);
  int *s_item = reinterpret_cast<int *>(smem + 64);
  if (threadIdx.x == 0) ws_init_barriers(smem, nbuf, WT * WD, kWsProdWarps);
  int jbase = 0;
  while (true) {
    if (threadIdx.x == 0) *s_item = atomicAdd(queue, 1);
    __syncthreads();
    const int it = *s_item;
    if (it >= nitems) break;
    const int4 w = items[it];           // {beam, DM tile, time tile, -}
    const WsBeam a = beams[w.x];
    const bool ok = ws_item<WT, WD, RD, uint8_t>(
        a, w.y, (int64_t)w.z * TT, jbase, smem, L, cc, nbuf, rawmax, elmax,
        err, timeout_cycles);
    jbase += (a.nchan + cc - 1) / cc;
    // every role is done with the item before the next one starts; a block
    // whose item failed stops taking work
    if (__syncthreads_or(!ok)) break;
  }
}

__global__ void batch_reset_kernel(int *queue, uint32_t *const *counts,
                                   int ncounts) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *queue = 0;
  if (i < ncounts) *counts[i] = 0;
}

template <int WT, int WD, int RD>
cudaError_t launch_persistent_t(const WsBeam *d_beams, const int4 *d_items,
                                int nitems, int *d_queue, int cc, int nbuf,
                                int rawmax, int elmax, size_t smem,
                                int32_t *d_err, int grid, cudaStream_t s) {
  auto kern = dedisp_persistent_kernel<WT, WD, RD>;
  static size_t attr_bytes = 0;
  if (smem > attr_bytes) {
    cudaError_t e = cudaFuncSetAttribute(
        kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_bytes = smem;
  }
  const long long timeout = 4000000000LL;  // ~2 s of SM clock
  kern<<<grid, 32 * (WT * WD + kWsProdWarps), smem, s>>>(
      d_beams, d_items, nitems, d_queue, cc, nbuf, rawmax, elmax, d_err,
      timeout);
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
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                             (int)smem);                                       \
    if (e == cudaSuccess)                                                      \
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(                       \
          &n, k, 32 * (WT_ * WD_ + kWsProdWarps), smem);                       \
  }
  DDSP_OCC(4, 2, 4) DDSP_OCC(2, 4, 4) DDSP_OCC(8, 1, 4)
  DDSP_OCC(4, 2, 8) DDSP_OCC(2, 4, 8) DDSP_OCC(8, 1, 8)
#undef DDSP_OCC
  return e == cudaSuccess ? n : 0;
}

cudaError_t launch_batch_reset(int *d_queue, uint32_t *const *d_counts,
                               int ncounts, cudaStream_t s) {
  const int n = ncounts > 1 ? ncounts : 1;
  batch_reset_kernel<<<(n + 255) / 256, 256, 0, s>>>(d_queue, d_counts,
                                                     ncounts);
  return cudaGetLastError();
}

cudaError_t launch_dedisperse_persistent(const DedispTile &t,
                                         const WsBeam *d_beams,
                                         const int4 *d_items, int nitems,
                                         int *d_queue, int rawmax, int elmax,
                                         size_t smem, int32_t *d_err, int grid,
                                         cudaStream_t s) {
#define DDSP_P(WT_, WD_, RD_)                                                 \
  if (t.wt == WT_ && t.wd == WD_ && t.rd == RD_)                              \
    return launch_persistent_t<WT_, WD_, RD_>(d_beams, d_items, nitems,       \
                                              d_queue, t.chan_chunk, t.nbuf,  \
                                              rawmax, elmax, smem, d_err,     \
                                              grid, s);
  DDSP_P(4, 2, 4) DDSP_P(2, 4, 4) DDSP_P(8, 1, 4)
  DDSP_P(4, 2, 8) DDSP_P(2, 4, 8) DDSP_P(8, 1, 8)
#undef DDSP_P
  return cudaErrorInvalidValue;
}

}  // namespace ddsp
