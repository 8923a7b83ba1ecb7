// peak.cu -- a measurement of this GPU's FP64 arithmetic rate
// (ibdvm_fp64_fma_rate), the roof against which the FP64 path is reported.
//
// The FP64 sweep is bound by the FP64 pipe rather than by HBM (a GB300 runs
// FP64 at a small fraction of its FP32 rate), so its roofline needs the rate
// this device sustains.  The kernel keeps eight independent FMA chains per
// thread in registers (no memory traffic in the timed loop), on enough blocks
// to fill every SM several times over, and is timed with CUDA events on the
// caller's stream after one untimed launch.  Flops count an FMA as two.
#include <cuda_runtime.h>

#include "ctx.h"

namespace ibdvm {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) fp64_fma_kernel(double *__restrict__ sink, int iters, double b) {
  double a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = 1e-3 * (threadIdx.x + j + 1);
  const double c = 1e-12;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (s == 12345.678) sink[blockIdx.x] = s; // keeps the chains alive; never true
}

} // namespace
} // namespace ibdvm

extern "C" ibdvm_status ibdvm_fp64_fma_rate(int iters, double *tflops, double *ms, void *cuda_stream) {
  if (iters <= 0 || !tflops) return IBDVM_E_INVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return IBDVM_E_CUDA;
  }
  const int blocks = 8 * nsm, threads = 256;
  double *sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ibdvm_status st = IBDVM_OK;
  float el = 0.f;
  if (cudaMalloc(&sink, blocks * sizeof(double)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    st = IBDVM_E_CUDA;
  } else {
    ibdvm::fp64_fma_kernel<<<blocks, threads, 0, s>>>(sink, iters / 4 + 1, 1.0000001); // untimed
    cudaEventRecord(e0, s);
    ibdvm::fp64_fma_kernel<<<blocks, threads, 0, s>>>(sink, iters, 1.0000001);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&el, e0, e1) != cudaSuccess || el <= 0.f)
      st = IBDVM_E_CUDA;
  }
  if (st == IBDVM_OK) {
    const double flops = 2.0 * 4.0 * ibdvm::kChains * static_cast<double>(iters) * blocks * threads;
    *tflops = flops / (el * 1e-3) / 1e12;
    if (ms) *ms = el;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  cudaGetLastError();
  return st;
}
