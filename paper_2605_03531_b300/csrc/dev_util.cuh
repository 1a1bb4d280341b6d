// dev_util.cuh -- device helpers shared by the dedispersion kernels: shared
// addresses, mbarriers with bounded waits, 1-D TMA bulk copies, named
// barriers, and the byte relayout that builds interleaved elements.
#pragma once

#include <stdint.h>

namespace ddsp {

// Bounds-checked build (compiled with -DDDSP_BOUNDS_CHECK and relocatable
// device code): a checked access first tests its index against the extent
// of its buffer; a failing test records (site << 32 | the index's low 32
// bits) as the library's first violation, if none is recorded yet
// (ddsp_bounds_check_status reads it), and the access is skipped.  In the
// normal build a check is the constant true and its expression is not
// evaluated.
#ifdef DDSP_BOUNDS_CHECK
extern __device__ unsigned long long g_bounds_first;
__device__ __forceinline__ bool bounds_ok(bool ok, uint32_t site,
                                          int64_t index) {
  if (!ok)
    atomicCAS(&g_bounds_first, 0ull,
              ((unsigned long long)site << 32) | (uint32_t)index);
  return ok;
}
#define DDSP_BC(cond, site, index) \
  (::ddsp::bounds_ok((cond), (site), (int64_t)(index)))
#else
#define DDSP_BC(cond, site, index) true
#endif

// Sites of the checks (the high word of a recorded violation).
enum : uint32_t {
  kBcSpsLoad = 101,     // series sample inside its row
  kBcSpsBuf = 102,      // window buffer (shared)
  kBcSpsScan = 103,     // scan group inside the buffer
  kBcSpsStats = 104,    // chunk statistics (shared)
  kBcSpsBound = 105,    // chunk read by the screen's bound
  kBcSpsQ = 106,        // prefix value read by the exact screen
  kBcSpsDense = 107,    // dense output inside its row
  kBcIlSrc = 201,       // interleaved row window of a bulk copy
  kBcIlDst = 202,       // bulk copy inside its channel's element stage
  kBcIlRel = 203,       // offsets copy inside its stage slot
  kBcIlElem = 204,      // consumer element reads inside the channel's stage
  kBcIlOut = 205,       // output sample inside the output row
  kBcStageIn = 301,     // spectra vector load inside the row
  kBcStageOut = 302,    // interleaved row store inside the row
  kBcIntlvIn = 303,     // channel-major (ring) read inside the row
  kBcIntlvOut = 304,    // interleaved store inside the row
  kBcUnpackIn = 305,    // spectra load inside the block
  kBcUnpackOut = 306,   // channel-major store inside the row
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile(
      "mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
          smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src,
                                         uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// One test of an mbarrier phase (the hardware may hold the thread a while
// before answering no).
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(a), "r"(parity)
      : "memory");
  return done != 0;
}

// One test that lets the hardware suspend the thread until the phase
// completes or about `hint_ns` pass, so a long wait costs a few polls of
// shared memory instead of one every few cycles.
__device__ __forceinline__ bool mbar_try_sleep(uint32_t a, uint32_t parity,
                                               uint32_t hint_ns) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(a), "r"(parity), "r"(hint_ns)
      : "memory");
  return done != 0;
}

// Bounded wait on an mbarrier phase: false if `limit` cycles pass first.
// A phase that is already complete costs one test and no clock read; later
// tests suspend the thread (up to 20 us each) until the phase completes.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          long long limit) {
  const uint32_t a = smem_u32(bar);
  if (mbar_try(a, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try_sleep(a, parity, 20000u)) return true;
    if (clock64() - t0 > limit) return false;
  }
}

// 4 raw words holding samples i..i+3 at stride S (rows m = 0..3) into the
// 4 interleaved elements i..i+3, element i = {x[i], x[i+S], x[i+2S],
// x[i+3S]} (byte m = row m): a 4x4 byte transpose.
__device__ __forceinline__ uint4 transpose4x4(uint32_t r0, uint32_t r1,
                                              uint32_t r2, uint32_t r3) {
  const uint32_t t0 = __byte_perm(r0, r1, 0x5140);
  const uint32_t t1 = __byte_perm(r0, r1, 0x7362);
  const uint32_t t2 = __byte_perm(r2, r3, 0x5140);
  const uint32_t t3 = __byte_perm(r2, r3, 0x7362);
  uint4 o;
  o.x = __byte_perm(t0, t2, 0x5410);
  o.y = __byte_perm(t0, t2, 0x7632);
  o.z = __byte_perm(t1, t3, 0x5410);
  o.w = __byte_perm(t1, t3, 0x7632);
  return o;
}

}  // namespace ddsp
