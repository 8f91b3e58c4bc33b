// Asynchronous-copy pipeline primitives shared by the H * V kernels: mbarriers with bounded waits
// (%globaltimer) and bulk global -> shared copies that complete on an mbarrier.
#pragma once
#include <cstdint>

namespace css_pipe {

constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s per wait

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void bar_expect(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_test(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the phase of `parity`; gives up when the CTA's abort flag is set or after
// limit_ns (then sets the abort flag and the error flag)
__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag, int* err,
                                         uint64_t limit_ns = kWaitNs) {
  if (bar_test(b, parity)) return true;
  const uint64_t t0 = gtime();
  for (uint32_t it = 1;; ++it) {
    if (bar_test(b, parity)) return true;
    if ((it & 255) == 0) {
      if (*abort_flag) return false;
      if (gtime() - t0 > limit_ns) {
        *abort_flag = 1;
        atomicOr(err, 1);
        return false;
      }
    }
  }
}
// the same without abort: used at tear-down for copies that are already in flight
__device__ __forceinline__ void bar_drain(uint64_t* b, uint32_t parity, uint64_t limit_ns = kWaitNs) {
  const uint64_t t0 = gtime();
  while (!bar_test(b, parity))
    if (gtime() - t0 > limit_ns) return;
}
// bytes (a multiple of 16, both addresses 16-byte aligned) from global to shared memory,
// completing on mbarrier b (which must expect them)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   su32(dst)),
               "l"(src), "r"(bytes), "r"(su32(b))
               : "memory");
}

}  // namespace css_pipe
