// Cooperative launch of the persistent MGS kernel (all CTAs co-resident: the kernel's
// grid barriers and pivot flags rely on it).
#pragma once

#include <cuda_runtime.h>

#include "mgs_kernel.cuh"

namespace mgs {

template <class Ar>
int launch_kernel(const Params& pr, int grid, size_t smem, cudaStream_t stream) {
  auto kern = mgs_ls_kernel<Ar>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  if (e != cudaSuccess) return (int)e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (per_sm * sms < grid) return (int)cudaErrorCooperativeLaunchTooLarge;
  Params copy = pr;
  void* args[] = {&copy};
  e = cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(kThreads), args, smem, stream);
  return (int)e;
}

int launch_d(const Params& pr, int grid, size_t smem, cudaStream_t stream);
int launch_dd(const Params& pr, int grid, size_t smem, cudaStream_t stream);
int launch_qd(const Params& pr, int grid, size_t smem, cudaStream_t stream);

}  // namespace mgs
