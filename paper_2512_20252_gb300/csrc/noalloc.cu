// noalloc.cu -- a residual entry point that allocates no device memory.
//
// Some callers cannot allocate device memory at the moment they need the
// steady-state residual: code that runs while another runtime owns the whole
// device-memory pool and forbids cudaMalloc, hosts that must keep a fixed
// memory footprint after start-up, and work enqueued between other launches
// where cudaMalloc / cudaFree would synchronise the device and stall the
// overlap.  ibdvm_residual_noalloc serves them: it computes the same residual
// as ibdvm_step reports, from two conservative-variable fields the caller
// already holds on the device, and keeps its per-block partial sums in a
// fixed array compiled into the library instead of allocated memory.
//
// The array is a file-scope __device__ symbol of kMaxBlocks * 2 * 5 doubles
// (640 KiB); every GPU that loads the library reserves it until the process
// exits.  Host code cannot use the symbol's name as a device address, so the
// first call in each CUDA context (the context current at the call: the
// device's primary context for runtime-API callers, or a context the caller
// made current with the driver API) looks the address up with
// cudaGetSymbolAddress and caches it under that context's handle; make that
// first call before any stream capture.  A context that is destroyed and
// replaced by a new one with the same handle is not detected: after
// cudaDeviceReset, a caller that keeps using this entry point makes its first
// call again outside any capture.  All calls share the array and it keeps the last call's
// partial sums: every block overwrites its own slots before they are read, so
// nothing needs clearing, but two calls that overlap on the GPU (different
// streams, or different host threads) race on it and must be serialised by
// the caller.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/ibdvm.h"

namespace ibdvm {
void set_thread_error(const std::string &e); // capi.cpp: message for ibdvm_last_error(NULL)
}

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 8192;                  // at most kMaxBlocks * kThreads cells per call
constexpr long long kMaxCells = static_cast<long long>(kMaxBlocks) * kThreads; // 2,097,152
constexpr int kMaxW = 5;                          // conservative variables in 3D
constexpr int kMaxContexts = 64;

// per-block sums of (dW_i)^2 and |W_i|, [block][2 * NW]
static __device__ __align__(256) double g_residual_scratch[kMaxBlocks * 2 * kMaxW];

std::mutex g_mu;
// the array's address in each context met so far
struct CtxAddr {
  CUcontext ctx;
  double *addr;
};
CtxAddr g_scratch_addr[kMaxContexts] = {};
int g_nctx = 0;

// the current CUDA context through the driver entry point (no link to libcuda)
CUresult current_context(CUcontext *out) {
  using Fn = CUresult (*)(CUcontext *);
  static Fn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return CUDA_ERROR_NOT_SUPPORTED;
    fn = reinterpret_cast<Fn>(p);
  }
  return fn(out);
}

template <int NW>
__global__ void __launch_bounds__(kThreads)
residual_partials(const double *__restrict__ Wold, const double *__restrict__ Wnew,
                  const unsigned char *__restrict__ ctype, long long ncell, double *__restrict__ scratch) {
  __shared__ double red[2 * NW][kThreads / 32];
  const long long c = static_cast<long long>(blockIdx.x) * kThreads + threadIdx.x;
  double num[NW], den[NW];
#pragma unroll
  for (int i = 0; i < NW; ++i) num[i] = den[i] = 0.0;
  if (c < ncell && (ctype == nullptr || ctype[c] == IBDVM_CELL_FLUID)) {
#pragma unroll
    for (int i = 0; i < NW; ++i) {
      const double wn = Wnew[c * NW + i];
      const double d = wn - Wold[c * NW + i];
      num[i] = d * d;
      den[i] = fabs(wn);
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NW; ++i) {
    double a = num[i], b = den[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
      red[i][wid] = a;
      red[NW + i][wid] = b;
    }
  }
  __syncthreads();
  if (threadIdx.x < 2 * NW) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += red[threadIdx.x][w];
    scratch[static_cast<size_t>(blockIdx.x) * 2 * NW + threadIdx.x] = s;
  }
}

template <int NW>
__global__ void residual_combine(const double *__restrict__ scratch, int nblk, double *__restrict__ out) {
  __shared__ double sh[kThreads];
  __shared__ double tot[2 * NW];
  for (int i = 0; i < 2 * NW; ++i) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += kThreads) s += scratch[static_cast<size_t>(b) * 2 * NW + i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) tot[i] = sh[0];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int i = 0; i < NW; ++i) {
      if (tot[NW + i] == 0.0) continue; // a component that is zero everywhere does not count
      const double v = sqrt(tot[i]) / tot[NW + i];
      r = (v > r) ? v : r;
    }
    *out = r;
  }
}

ibdvm_status fail(const std::string &msg, ibdvm_status st) {
  ibdvm::set_thread_error(msg);
  return st;
}

} // namespace

extern "C" ibdvm_status ibdvm_residual_noalloc(const double *W_old, const double *W_new,
                                               const unsigned char *celltype, long long ncell, int dim,
                                               double *residual, void *cuda_stream) {
  if (!W_old || !W_new || !residual) return fail("residual_noalloc: a required pointer is NULL", IBDVM_E_INVAL);
  if (dim != 2 && dim != 3) return fail("residual_noalloc: dim must be 2 or 3", IBDVM_E_INVAL);
  if (ncell < 1 || ncell > kMaxCells)
    return fail("residual_noalloc: ncell = " + std::to_string(ncell) + " is outside [1, " +
                    std::to_string(kMaxCells) + "], the capacity of the built-in scratch array",
                IBDVM_E_INVAL);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(std::string("residual_noalloc: cudaGetDevice: ") + cudaGetErrorString(e), IBDVM_E_CUDA);
  CUcontext ctx = nullptr;
  if (current_context(&ctx) != CUDA_SUCCESS) return fail("residual_noalloc: cuCtxGetCurrent failed", IBDVM_E_CUDA);
  if (!ctx) {
    // no context current yet: make the device's primary context current
    e = cudaSetDevice(dev);
    if (e != cudaSuccess || current_context(&ctx) != CUDA_SUCCESS || !ctx)
      return fail("residual_noalloc: no CUDA context could be made current", IBDVM_E_CUDA);
  }
  double *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    for (int i = 0; i < g_nctx && !scratch; ++i)
      if (g_scratch_addr[i].ctx == ctx) scratch = g_scratch_addr[i].addr;
    if (!scratch) {
      if (g_nctx == kMaxContexts) return fail("residual_noalloc: more than 64 CUDA contexts", IBDVM_E_INVAL);
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_residual_scratch);
      if (e != cudaSuccess)
        return fail(std::string("residual_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e), IBDVM_E_CUDA);
      scratch = static_cast<double *>(p);
      g_scratch_addr[g_nctx++] = CtxAddr{ctx, scratch};
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int nblk = static_cast<int>((ncell + kThreads - 1) / kThreads);
  if (dim == 2) {
    residual_partials<4><<<nblk, kThreads, 0, s>>>(W_old, W_new, celltype, ncell, scratch);
    residual_combine<4><<<1, kThreads, 0, s>>>(scratch, nblk, residual);
  } else {
    residual_partials<5><<<nblk, kThreads, 0, s>>>(W_old, W_new, celltype, ncell, scratch);
    residual_combine<5><<<1, kThreads, 0, s>>>(scratch, nblk, residual);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(std::string("residual_noalloc: launch: ") + cudaGetErrorString(e), IBDVM_E_CUDA);
  return IBDVM_OK;
}
