// k_unpack.cu -- step 2 of the path: time-major spectra (a block of spectra,
// one row of nchan samples per time sample, Sec.2.2) to channel-major rows
// so the dedispersion kernel can stage a channel's time series with one
// contiguous bulk copy.  HBM-bound: every byte is read once and written once.
// Each row gets columns [0, ncols) (ncols <= pitch): input samples, then
// zeros past nsamp_in; columns from ncols to the pitch are left untouched.
#include "dev_util.cuh"
#include "internal.h"

namespace ddsp {
namespace {

// uint8, nchan % 16 == 0: 128 samples x 128 channels per block.  Loads are
// 16-byte vectors along channels; the transpose is done on 4x4 byte blocks
// with byte permutes so that stores are 4-byte words along time.
constexpr int kTS = 128;            // samples per tile
constexpr int kTC = 128;            // channels per tile
constexpr int kPitchW = kTC / 4 + 1; // smem row pitch in words (bank skew)

__device__ __forceinline__ void unpack_u8_tile(
    const uint8_t *__restrict__ in, int64_t nsamp_in, int nchan,
    uint8_t *__restrict__ out, int64_t pitch, int64_t ncols, int64_t tile_s,
    int tile_c) {
  __shared__ uint32_t tile[kTS * kPitchW];
  const int tid = threadIdx.x;
  const int64_t s0 = tile_s * kTS;
  const int c0 = tile_c * kTC;
  // ---- load: 128 rows x 8 16-byte vectors
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int idx = tid + 256 * i;
    int row = idx >> 3, q = idx & 7;
    int64_t s = s0 + row;
    int c = c0 + 16 * q;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (s < nsamp_in && c < nchan && DDSP_BC(c + 16 <= nchan, kBcUnpackIn, c))
      v = __ldg(reinterpret_cast<const uint4 *>(in + s * nchan + c));
    uint32_t *dst = tile + row * kPitchW + 4 * q;
    dst[0] = v.x; dst[1] = v.y; dst[2] = v.z; dst[3] = v.w;
  }
  __syncthreads();
  // ---- transpose 4x4 byte blocks and store channel-major
  const int lane = tid & 31, w = tid >> 5;
  const int sq = (lane & 7) + 8 * (w & 3);
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    int cq = (lane >> 3) + 4 * (w >> 2) + 8 * it;
    const uint32_t *src = tile + (4 * sq) * kPitchW + cq;
    uint32_t r0 = src[0], r1 = src[kPitchW], r2 = src[2 * kPitchW],
             r3 = src[3 * kPitchW];
    uint32_t t0 = __byte_perm(r0, r1, 0x5140), t1 = __byte_perm(r0, r1, 0x7362);
    uint32_t t2 = __byte_perm(r2, r3, 0x5140), t3 = __byte_perm(r2, r3, 0x7362);
    uint32_t o[4] = {__byte_perm(t0, t2, 0x5410), __byte_perm(t0, t2, 0x7632),
                     __byte_perm(t1, t3, 0x5410), __byte_perm(t1, t3, 0x7632)};
    int64_t s = s0 + 4 * sq;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int c = c0 + 4 * cq + j;
      if (c < nchan && s < ncols && DDSP_BC(s + 4 <= pitch, kBcUnpackOut, s))
        *reinterpret_cast<uint32_t *>(out + (int64_t)c * pitch + s) = o[j];
    }
  }
}

__global__ void __launch_bounds__(256)
unpack_u8_kernel(const uint8_t *__restrict__ in, int64_t nsamp_in, int nchan,
                 uint8_t *__restrict__ out, int64_t pitch, int64_t ncols) {
  unpack_u8_tile(in, nsamp_in, nchan, out, pitch, ncols, blockIdx.x,
                 blockIdx.y);
}

// Generic element-wise transpose (uint8 with nchan % 16 != 0, and uint16):
// 32 x 32 elements per block through a skewed shared tile.
template <typename T>
__global__ void __launch_bounds__(256)
unpack_generic_kernel(const T *__restrict__ in, int64_t nsamp_in, int nchan,
                      T *__restrict__ out, int64_t pitch, int64_t ncols) {
  __shared__ T tile[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const int64_t s0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
#pragma unroll
  for (int r = ty; r < 32; r += 8) {
    int64_t s = s0 + r;
    int c = c0 + tx;
    T v = 0;
    if (s < nsamp_in && c < nchan) v = in[s * nchan + c];
    tile[r][tx] = v;
  }
  __syncthreads();
#pragma unroll
  for (int r = ty; r < 32; r += 8) {
    int c = c0 + r;
    int64_t s = s0 + tx;
    if (c < nchan && s < ncols && DDSP_BC(s < pitch, kBcUnpackOut, s))
      out[(int64_t)c * pitch + s] = tile[tx][r];
  }
}

}  // namespace

cudaError_t launch_unpack_cols(const void *d_in, int64_t nsamp_in, int nchan,
                               int nbits, void *d_out, int64_t pitch,
                               int64_t ncols, cudaStream_t s) {
  if (ncols > pitch || ncols < 0) return cudaErrorInvalidValue;
  if (ncols == 0) return cudaSuccess;
  if (nbits == 8 && nchan % 16 == 0) {
    if (ncols % 4) return cudaErrorInvalidValue;  // 4-sample word stores
    dim3 grid((unsigned)((ncols + kTS - 1) / kTS),
              (unsigned)((nchan + kTC - 1) / kTC));
    unpack_u8_kernel<<<grid, 256, 0, s>>>(static_cast<const uint8_t *>(d_in),
                                          nsamp_in, nchan,
                                          static_cast<uint8_t *>(d_out), pitch,
                                          ncols);
  } else if (nbits == 8) {
    dim3 grid((unsigned)((ncols + 31) / 32), (unsigned)((nchan + 31) / 32));
    unpack_generic_kernel<uint8_t><<<grid, 256, 0, s>>>(
        static_cast<const uint8_t *>(d_in), nsamp_in, nchan,
        static_cast<uint8_t *>(d_out), pitch, ncols);
  } else {
    dim3 grid((unsigned)((ncols + 31) / 32), (unsigned)((nchan + 31) / 32));
    unpack_generic_kernel<uint16_t><<<grid, 256, 0, s>>>(
        static_cast<const uint16_t *>(d_in), nsamp_in, nchan,
        static_cast<uint16_t *>(d_out), pitch, ncols);
  }
  return cudaGetLastError();
}

cudaError_t launch_unpack(const void *d_in, int64_t nsamp_in, int nchan,
                          int nbits, void *d_out, int64_t pitch,
                          cudaStream_t s) {
  return launch_unpack_cols(d_in, nsamp_in, nchan, nbits, d_out, pitch, pitch,
                            s);
}

}  // namespace ddsp
