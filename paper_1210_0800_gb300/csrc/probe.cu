// Two probes with no counterpart in the paper.
//
// FP64 FMA throughput probe: the rate the roofline of the FP64-bound solve divides by.
// Every thread runs eight independent multiply-add chains (enough independent work to keep
// the FP64 unit of its SM sub-partition busy); the result is written so that nothing can be
// elided.
//
// Wait probe: one of the solver kernels' bounded waits (the pivot-flag wait, the grid
// barrier) on a condition that never comes true, so that it runs out of time; the host
// then reads the status and the abort flag the wait left.  Failure detection is checked
// this way without faulting or hanging the GPU.
#include <cuda_runtime.h>

#include "../../include/mgs_ddqd.h"
#include "mgs_kernel.cuh"

namespace {

__global__ void fp64_fma_probe(double* out, int iters, double a, double b) {
  double x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (int i = 0; i < iters; ++i) {
    x0 = __fma_rn(x0, a, b);
    x1 = __fma_rn(x1, a, b);
    x2 = __fma_rn(x2, a, b);
    x3 = __fma_rn(x3, a, b);
    x4 = __fma_rn(x4, a, b);
    x5 = __fma_rn(x5, a, b);
    x6 = __fma_rn(x6, a, b);
    x7 = __fma_rn(x7, a, b);
  }
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
}

// words: [0] arrival counter, [1] abort flag, [2] status, [3] a flag nothing sets.
__global__ void wait_probe_kernel(unsigned* words, int kind, long long timeout_ns) {
  mgs::Params pr{};
  pr.sync = words;
  pr.status = reinterpret_cast<int*>(words + 2);
  pr.timeout_ns = timeout_ns;
  if (kind == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) mgs::wait_flag(pr, reinterpret_cast<const int*>(words + 3));
  } else if (blockIdx.x == 0) {  // kind 1: CTA 1 of 2 never arrives at the barrier
    unsigned epoch = 0;
    mgs::grid_barrier(pr, epoch);
  }
}

}  // namespace

extern "C" int mgs_wait_probe(unsigned* dev_words, int kind, long long timeout_ns, void* stream) {
  if (!dev_words || (reinterpret_cast<uintptr_t>(dev_words) & 3u) || (kind != 0 && kind != 1) || timeout_ns < 1 ||
      timeout_ns > 10000000000LL)
    return MGS_EINVAL;
  wait_probe_kernel<<<kind == 0 ? 1 : 2, 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(dev_words, kind, timeout_ns);
  return cudaGetLastError() == cudaSuccess ? MGS_OK : MGS_ECUDA;
}

extern "C" int mgs_fp64_probe(double* dev_out, int blocks, int threads, int iters, void* stream) {
  if (!dev_out || blocks < 1 || threads < 32 || threads > 1024 || (threads & 31) || iters < 1) return MGS_EINVAL;
  fp64_fma_probe<<<blocks, threads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(dev_out, iters, 0.999999, 1e-7);
  return cudaGetLastError() == cudaSuccess ? MGS_OK : MGS_ECUDA;
}
