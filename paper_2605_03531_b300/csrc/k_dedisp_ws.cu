// k_dedisp_ws.cu -- warp-specialised brute-force dedispersion (Sec.3.2) of
// one plan: one block per (DM tile, time tile), running one work item of
// ws_item.cuh.  Producer warps stage and relayout, consumer warps
// accumulate; they overlap through mbarriers with no block-wide barrier in
// the main loop.
#include "ws_item.cuh"

namespace ddsp {
namespace {

template <int WT, int WD, int RD, typename T>
__global__ void __launch_bounds__(32 * (WT * WD + kWsProdWarps), 2)
dedisp_ws_kernel(WsBeam a, int nbuf, int32_t *err, long long timeout_cycles) {
  constexpr int SPE = 4 / sizeof(T);
  constexpr int TT = SPE * 32 * kElemPerThread * WT;
  extern __shared__ __align__(16) unsigned char smem[];
  if (threadIdx.x == 0) ws_init_barriers(smem, nbuf, WT * WD);
  __syncthreads();
  ws_item<WT, WD, RD, T>(a, blockIdx.x, (int64_t)blockIdx.y * TT, 0, smem,
                         nbuf, err, timeout_cycles);
}

template <int WT, int WD, int RD, typename T>
cudaError_t launch_ws_t(const Plan &p, const void *d_cm, int64_t pitch,
                        int64_t nsamp_out, int32_t *d_out, cudaStream_t s,
                        int rawmax, int elmax, size_t smem) {
  auto kern = dedisp_ws_kernel<WT, WD, RD, T>;
  {
    cudaError_t e = smem_opt_in(kern);
    if (e != cudaSuccess) return e;
  }
  constexpr int SPE = 4 / sizeof(T);
  constexpr int TT = SPE * 32 * kElemPerThread * WT;
  const int ntt = (int)((nsamp_out + TT - 1) / TT);
  WsBeam a{};
  a.cm = d_cm;
  a.pitch = pitch;
  a.nsamp_out = nsamp_out;
  a.ring = 0;
  a.t0 = 0;
  a.out_pitch = nsamp_out;
  a.desc = reinterpret_cast<const int2 *>(p.tab.d_desc);
  a.relb = p.tab.d_relb;
  a.rowmap = p.tab.d_rowmap;
  a.out = d_out;
  a.nchan = p.nchan;
  a.n_dm_tiles = p.tab.n_dm_tiles;
  a.n_time_tiles = ntt;
  a.cc = p.tile.chan_chunk;
  a.rawmax = rawmax;
  a.elmax = elmax;
  dim3 grid((unsigned)p.tab.n_dm_tiles, (unsigned)ntt);
  const long long timeout = 4000000000LL;  // ~2 s of SM clock
  kern<<<grid, 32 * (WT * WD + kWsProdWarps), smem, s>>>(
      a, p.tile.nbuf, p.d_err, timeout);
  return cudaGetLastError();
}

}  // namespace

size_t dedisp_ws_smem_bytes(int chan_chunk, int dm_tile, int rawmax,
                            int elmax, int nbuf) {
  return (size_t)WsLayout(chan_chunk, dm_tile, rawmax, elmax, nbuf).total;
}

cudaError_t launch_dedisperse_ws(const Plan &p, const void *d_cm,
                                 int64_t pitch, int64_t nsamp_out,
                                 int32_t *d_out, cudaStream_t s, int rawmax,
                                 int elmax, size_t smem) {
  const int wt = p.tile.wt, wd = p.tile.wd, rd = p.tile.rd;
#define DDSP_WS(WT_, WD_, RD_, T_)                                          \
  if (wt == WT_ && wd == WD_ && rd == RD_)                                  \
    return launch_ws_t<WT_, WD_, RD_, T_>(p, d_cm, pitch, nsamp_out, d_out, \
                                          s, rawmax, elmax, smem);
  if (p.nbits == 8) {
    DDSP_WS(4, 2, 4, uint8_t)
    DDSP_WS(2, 4, 4, uint8_t)
    DDSP_WS(8, 1, 4, uint8_t)
    DDSP_WS(4, 2, 8, uint8_t)
    DDSP_WS(2, 4, 8, uint8_t)
    DDSP_WS(8, 1, 8, uint8_t)
  } else {
    DDSP_WS(4, 2, 4, uint16_t)
    DDSP_WS(2, 4, 4, uint16_t)
    DDSP_WS(8, 1, 4, uint16_t)
  }
#undef DDSP_WS
  return cudaErrorInvalidValue;
}

}  // namespace ddsp
