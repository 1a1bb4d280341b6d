// k_probe.cu -- microbenchmarks of the two on-chip units the dedispersion
// kernels are bound by (Sec.3.2 is integer adds of bytes read from shared
// memory): 32-bit shared-memory load bandwidth, the integer ALU rate of the
// two instructions the SWAR accumulation uses (3-input add, byte permute),
// and the dedispersion inner loop itself on data resident in shared memory
// (no staging, no synchronisation).  Each kernel runs a wave of identical
// blocks (SMs x resident blocks); every block records its SM and the clock64
// values around its loop, and an SM's rate is the work of its blocks over
// the span from their first start to their last end (clock64 is per SM),
// whatever number of blocks actually shared the SM.
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "host.h"

namespace ddsp {
namespace {

constexpr int kProbeThreads = 512;
constexpr int kProbeWords = 8192;   // 32 KB of shared memory

// Block b's {SM id, loop start, loop end} (clock64 of that SM).
__device__ __forceinline__ void record(long long *rec, long long t0,
                                       long long t1) {
  uint32_t smid;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
  rec[3 * blockIdx.x] = smid;
  rec[3 * blockIdx.x + 1] = t0;
  rec[3 * blockIdx.x + 2] = t1;
}

// 16 conflict-free 32-bit loads per thread and iteration (consecutive lanes,
// consecutive words), folded into 2 accumulators by 3-input XORs.
__global__ void __launch_bounds__(kProbeThreads)
probe_smem_kernel(int iters, uint32_t *sink, long long *cycles) {
  __shared__ uint32_t buf[kProbeWords];
  for (int i = threadIdx.x; i < kProbeWords; i += blockDim.x)
    buf[i] = (uint32_t)i * 2654435761u;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t a0 = 0, a1 = 0;
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
    asm volatile("" ::: "memory");
    // 16 rows of 512 words; the base (< 512 words) rotates per warp and
    // iteration; the largest index is 511 + 512 * 12 + 1536 = 8191
    const uint32_t *q = buf + lane + ((warp + it) & 15) * 32;
#pragma unroll
    for (int k = 0; k < 16; k += 4) {
      a0 ^= q[512 * k] ^ q[512 * k + 512];
      a1 ^= q[512 * k + 1024] ^ q[512 * k + 1536];
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  if (threadIdx.x == 0) record(cycles, t0, t1);
  sink[blockIdx.x * blockDim.x + threadIdx.x] = a0 ^ a1;
}

// 8 chains per thread of the instruction under test; each step also reads
// the next chain's value, so the compiler cannot fold repeated steps.
template <int OP>   // 0: 3-input add, 1: byte permute
__global__ void __launch_bounds__(kProbeThreads)
probe_alu_kernel(int iters, uint32_t seed, uint32_t *sink, long long *cycles) {
  uint32_t a[8], b[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    a[k] = seed * (threadIdx.x + 1) + k;
    b[k] = seed ^ (k * 0x9E3779B9u);
  }
  __syncthreads();
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (OP == 0) a[k] = a[k] + a[(k + 1) & 7] + b[k];
        else a[k] = __byte_perm(a[k], a[(k + 1) & 7], 0x6351 + r);
      }
  }
  __syncthreads();
  const long long t1 = clock64();
  if (threadIdx.x == 0) record(cycles, t0, t1);
  uint32_t x = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) x ^= a[k];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = x;
}

// The dedispersion consumer loop as the default tile runs it (4 DM trials x
// 8 elements per thread, 16 warps as 4 along time x 4 along DM, two
// channels per step: per pair of words two 32-bit loads, one 3-input add,
// two byte permutes and two multiply-adds by `one` on the FMA pipe) over 4
// resident channels of 2048 elements with fixed delay offsets: the ceiling
// of the inner loop with no staging and no handoff.
__global__ void __launch_bounds__(kProbeThreads)
probe_swar_kernel(int iters, uint32_t one, uint32_t *sink, long long *cycles) {
  constexpr int RD = 4, E = 8, NQ = 4, EL = 2048;
  __shared__ uint32_t elem[NQ * EL];   // 32 KB
  __shared__ int rel[NQ * 16];
  for (int i = threadIdx.x; i < NQ * EL; i += blockDim.x)
    elem[i] = (uint32_t)i * 2654435761u;
  for (int i = threadIdx.x; i < NQ * 16; i += blockDim.x)
    rel[i] = 4 * ((i % 16) * 37 % 480);   // offsets below 480 elements
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wt = warp & 3, wd = warp >> 2;   // 4 x 4 warps
  const unsigned char *eb =
      reinterpret_cast<const unsigned char *>(elem) + 4 * (256 * wt + lane);
  uint32_t A[RD][E], B[RD][E];
#pragma unroll
  for (int r = 0; r < RD; ++r)
#pragma unroll
    for (int e = 0; e < E; ++e) A[r][e] = B[r][e] = 0;
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
    // reload every iteration, a few bytes further along: the largest byte
    // address in a channel is 4*479 + 4*(768+31) + 128*7 + 28 = 6036 < 4*EL
    asm volatile("" ::: "memory");
    const unsigned char *ei = eb + 4 * (it & 7);
    for (int q = 0; q < NQ; q += 2) {
      int ra[RD], rb[RD];
      const int4 x = *reinterpret_cast<const int4 *>(rel + q * 16 + RD * wd);
      const int4 y = *reinterpret_cast<const int4 *>(rel + (q + 1) * 16 + RD * wd);
      ra[0] = x.x; ra[1] = x.y; ra[2] = x.z; ra[3] = x.w;
      rb[0] = y.x; rb[1] = y.y; rb[2] = y.z; rb[3] = y.w;
      const unsigned char *ea = ei + q * EL * 4, *eb2 = ea + EL * 4;
#pragma unroll
      for (int r = 0; r < RD; ++r)
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const uint32_t wa = *reinterpret_cast<const uint32_t *>(ea + ra[r] + 128 * e);
          const uint32_t wb = *reinterpret_cast<const uint32_t *>(eb2 + rb[r] + 128 * e);
          A[r][e] += wa + wb;
          B[r][e] = __byte_perm(wa, 0u, 0x4341) * one + B[r][e];
          B[r][e] = __byte_perm(wb, 0u, 0x4341) * one + B[r][e];
        }
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  if (threadIdx.x == 0) record(cycles, t0, t1);
  uint32_t x = 0;
#pragma unroll
  for (int r = 0; r < RD; ++r)
#pragma unroll
    for (int e = 0; e < E; ++e) x ^= A[r][e] ^ B[r][e];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = x;
}

// Median over SMs of (work of the SM's blocks) / (cycles from the first
// start to the last end among them).
double median_sm_rate(const long long *d_rec, int n, double work_per_block) {
  std::vector<long long> h(3 * (size_t)n);
  cudaMemcpy(h.data(), d_rec, h.size() * sizeof(long long),
             cudaMemcpyDeviceToHost);
  struct Span { long long lo, hi; int blocks; };
  std::vector<Span> sm;
  for (int b = 0; b < n; ++b) {
    const long long id = h[3 * b], t0 = h[3 * b + 1], t1 = h[3 * b + 2];
    if (id < 0 || id > 4096) continue;
    if ((size_t)id >= sm.size()) sm.resize(id + 1, Span{0, 0, 0});
    Span &x = sm[id];
    if (x.blocks == 0) x = Span{t0, t1, 0};
    x.lo = std::min(x.lo, t0);
    x.hi = std::max(x.hi, t1);
    ++x.blocks;
  }
  std::vector<double> rate;
  for (const Span &x : sm)
    if (x.blocks > 0 && x.hi > x.lo)
      rate.push_back(x.blocks * work_per_block / (double)(x.hi - x.lo));
  if (rate.empty()) return 0.0;
  std::sort(rate.begin(), rate.end());
  return rate[rate.size() / 2];
}

template <typename Kern, typename Launch>
int run_probe(Kern kern, Launch launch, int sms, int *blocks_per_sm,
              double work_per_block, uint32_t *d_sink, long long *d_cycles,
              double *rate) {
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &occ, kern, kProbeThreads, 0);
  if (e != cudaSuccess) return cuda_rc(e);
  if (occ < 1) return DDSP_E_CUDA;
  occ = std::min(occ, 8);      // the sink and cycle arrays hold 8 per SM
  const int grid = sms * occ;
  launch(grid, 1);            // warm-up
  launch(grid, 0);
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_rc(e);
  *blocks_per_sm = occ;
  *rate = median_sm_rate(d_cycles, grid, work_per_block);
  return *rate > 0.0 ? DDSP_OK : DDSP_E_CUDA;
}

}  // namespace
}  // namespace ddsp

using namespace ddsp;

extern "C" int ddsp_probe_unit_peaks(int device, ddsp_unit_peaks *out) {
  if (!out) return DDSP_E_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return DDSP_E_INVALID_ARG;
  DeviceGuard g(device);
  int sms = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount,
                                         device);
  if (e != cudaSuccess) return cuda_rc(e);
  *out = ddsp_unit_peaks{};
  out->sms = sms;
  const int maxgrid = sms * 8;
  uint32_t *d_sink = nullptr;
  long long *d_cycles = nullptr;
  if ((e = cudaMalloc(&d_sink, (size_t)maxgrid * kProbeThreads * 4)) !=
          cudaSuccess ||
      (e = cudaMalloc(&d_cycles, (size_t)maxgrid * 3 * sizeof(long long))) !=
          cudaSuccess) {
    cudaFree(d_sink);
    return cuda_rc(e);
  }
  const int it_smem = 4096, it_alu = 4096, it_swar = 512;
  int rc = run_probe(
      probe_smem_kernel,
      [&](int grid, int warm) {
        probe_smem_kernel<<<grid, kProbeThreads>>>(warm ? 16 : it_smem, d_sink,
                                                   d_cycles);
      },
      sms, &out->blocks_per_sm[0], (double)kProbeThreads * it_smem * 16 * 4,
      d_sink, d_cycles, &out->smem_bytes_per_clk);
  if (rc == DDSP_OK)
    rc = run_probe(
        probe_alu_kernel<0>,
        [&](int grid, int warm) {
          probe_alu_kernel<0><<<grid, kProbeThreads>>>(warm ? 16 : it_alu, 12345u,
                                                      d_sink, d_cycles);
        },
        sms, &out->blocks_per_sm[1], (double)kProbeThreads * it_alu * 32,
        d_sink, d_cycles, &out->iadd3_per_clk);
  if (rc == DDSP_OK)
    rc = run_probe(
        probe_alu_kernel<1>,
        [&](int grid, int warm) {
          probe_alu_kernel<1><<<grid, kProbeThreads>>>(warm ? 16 : it_alu, 12345u,
                                                      d_sink, d_cycles);
        },
        sms, &out->blocks_per_sm[2], (double)kProbeThreads * it_alu * 32,
        d_sink, d_cycles, &out->prmt_per_clk);
  if (rc == DDSP_OK)
    // per thread and iteration: 4 channels x 4 trials x 8 elements x 4 adds
    rc = run_probe(
        probe_swar_kernel,
        [&](int grid, int warm) {
          probe_swar_kernel<<<grid, kProbeThreads>>>(warm ? 4 : it_swar, 1u,
                                                     d_sink, d_cycles);
        },
        sms, &out->blocks_per_sm[3],
        (double)kProbeThreads * it_swar * 4 * 4 * 8 * 4, d_sink, d_cycles,
        &out->swar_adds_per_clk);
  cudaFree(d_sink);
  cudaFree(d_cycles);
  return rc;
}
