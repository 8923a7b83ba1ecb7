// selftest.cu -- a check of the bounded device waits (ibdvm_selftest_bounded_wait).
//
// The TMA-staged sweeps wait on mbarriers for their tile copies with a bound
// (tma_sync.cuh): when a copy does not arrive the block records a timeout and
// returns, and ibdvm_step reports IBDVM_E_TIMEOUT.  This kernel runs the same
// bounded wait on a barrier that expects 16 bytes: delivered by a bulk copy
// (the wait completes) or never delivered (nothing completes the phase, the
// wait runs out after `limit` polls and the kernel reports the timeout).  No
// copy is left in flight when the kernel returns.
#include <cuda_runtime.h>

#include <chrono>

#include "ctx.h"
#include "tma_sync.cuh"

namespace ibdvm {
namespace {

__global__ void bounded_wait_kernel(const float4 *__restrict__ src, int deliver, int limit, int *__restrict__ out) {
  __shared__ __align__(16) float4 buf;
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    buf = make_float4(0.f, 0.f, 0.f, 0.f);
    dev::mbar_init(&bar, 1);
    dev::fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    dev::fence_proxy_async();
    dev::mbar_expect_tx(&bar, 16);
    if (deliver)
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], 16, [%2];" ::"r"(
              dev::smem_addr(&buf)),
          "l"(reinterpret_cast<uint64_t>(src)), "r"(dev::smem_addr(&bar))
          : "memory");
  }
  const bool ok = dev::mbar_wait(&bar, 0, limit);
  const int timed_out = __syncthreads_or(ok ? 0 : 1);
  if (threadIdx.x == 0) {
    if (timed_out) out[0] = IBDVM_E_TIMEOUT;
    else out[0] = (buf.x == 1.f && buf.w == 4.f) ? IBDVM_OK : IBDVM_E_CUDA;
  }
}

} // namespace
} // namespace ibdvm

extern "C" ibdvm_status ibdvm_selftest_bounded_wait(int deliver, int spin_limit, double *seconds, void *cuda_stream) {
  if (spin_limit < 0 || spin_limit > ibdvm::dev::kSpinLimit) return IBDVM_E_INVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  void *mem = nullptr;
  if (cudaMalloc(&mem, 32) != cudaSuccess) {
    cudaGetLastError();
    return IBDVM_E_CUDA;
  }
  const float h[4] = {1.f, 2.f, 3.f, 4.f};
  int result = -1;
  const auto t0 = std::chrono::steady_clock::now();
  cudaError_t e = cudaMemcpyAsync(mem, h, sizeof(h), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    ibdvm::bounded_wait_kernel<<<1, 128, 0, s>>>(static_cast<const float4 *>(mem), deliver ? 1 : 0, spin_limit,
                                                 reinterpret_cast<int *>(static_cast<char *>(mem) + 16));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&result, static_cast<char *>(mem) + 16, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  const auto t1 = std::chrono::steady_clock::now();
  cudaFree(mem);
  if (seconds) *seconds = std::chrono::duration<double>(t1 - t0).count();
  if (e != cudaSuccess) {
    cudaGetLastError();
    return IBDVM_E_CUDA;
  }
  return static_cast<ibdvm_status>(result);
}
