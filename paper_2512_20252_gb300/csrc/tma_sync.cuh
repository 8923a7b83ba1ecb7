// tma_sync.cuh -- device helpers shared by the TMA-staged sweeps and the
// bounded-wait self-test: mbarrier set-up, arrive and bounded waits, proxy
// fences, and the packed FP32 van Leer face (Sec. 2.2, Eq. limiter).
//
// Every wait is bounded: mbar_wait polls try_wait at most `limit` more times
// and returns false instead of waiting on, so that a kernel can record a
// timeout, drain what it issued and return.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace ibdvm {
namespace dev {

constexpr int kSpinLimit = 1 << 18; // try_wait polls before a wait gives up (about 1 s: a poll suspends a few microseconds)

__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// one arrival that also expects `bytes` of asynchronous transfers on the barrier
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the phase of parity `parity` to complete: false after `limit` more polls
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, int limit = kSpinLimit) {
  if (mbar_try(bar, parity)) return true;
  for (int i = 0; i < limit; ++i)
    if (mbar_try(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float2 dup(float a) { return make_float2(a, a); }
// x - y for packed pairs, as one packed FMA
__device__ __forceinline__ float2 sub2(float2 x, float2 y) { return __ffma2_rn(y, make_float2(-1.f, -1.f), x); }
// Half the van Leer slope times the cell width for a pair of values, from the
// one-sided differences a = f - f_lo and b = f_hi - f (Eq. limiter):
// ab / (a + b) where a and b have the same sign, 0 otherwise.
__device__ __forceinline__ float2 vl_half2(float2 a, float2 b) {
  const float2 p = __fmul2_rn(a, b);
  const float2 s = __fadd2_rn(a, b);
  const float2 v = __fmul2_rn(p, make_float2(rcp_approx(s.x), rcp_approx(s.y)));
  return make_float2(p.x > 0.f ? v.x : 0.f, p.y > 0.f ? v.y : 0.f);
}
// Downwind face from the low and high neighbours and the packed sign s of the
// velocity: f + s vl(f - lo, hi - f), which equals f + vl(f - up, dn - f)
// because the half slope is symmetric in its arguments and odd.
__device__ __forceinline__ float2 face2(float2 f, float2 lo, float2 hi, float2 s) {
  return __ffma2_rn(s, vl_half2(sub2(f, lo), sub2(hi, f)), f);
}

} // namespace dev
} // namespace ibdvm
