// Cooperative launch of the persistent MGS kernel (all CTAs co-resident: the kernel's
// grid barriers and pivot flags rely on it).
#pragma once

#include <cuda_runtime.h>

#include "mgs_cluster.cuh"
#include "mgs_kernel.cuh"

namespace mgs {

// kind 0: mgs_ls_kernel (a grid barrier per step); kind 2: the cluster schedule with
// software groups (mgs_cluster_kernel<Ar, false>).
template <class Ar>
int launch_kernel(const Params& pr, int grid, size_t smem, cudaStream_t stream, int kind) {
  auto kern = kind == 2 ? mgs_cluster_kernel<Ar, false> : mgs_ls_kernel<Ar>;
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

// Cluster variant: clusters of `cl` CTAs (the row blocks of a column group).  Launched
// cooperatively when the driver accepts cooperative cluster launches, otherwise as a plain
// cluster launch after checking that every cluster can be resident at once.
template <class Ar>
int launch_cluster_kernel(const Params& pr, int grid, int cl, size_t smem, cudaStream_t stream) {
  auto kern = mgs_cluster_kernel<Ar, true>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attrs[2];
  attrs[0].id = cudaLaunchAttributeClusterDimension;
  attrs[0].val.clusterDim.x = cl;
  attrs[0].val.clusterDim.y = 1;
  attrs[0].val.clusterDim.z = 1;
  attrs[1].id = cudaLaunchAttributeCooperative;
  attrs[1].val.cooperative = 1;
  cfg.attrs = attrs;
  cfg.numAttrs = 1;
  int max_clusters = 0;
  e = cudaOccupancyMaxActiveClusters(&max_clusters, kern, &cfg);
  if (e != cudaSuccess) return (int)e;
  if (max_clusters * cl < grid) return (int)cudaErrorCooperativeLaunchTooLarge;
  Params copy = pr;
  cfg.numAttrs = 2;
  e = cudaLaunchKernelEx(&cfg, kern, copy);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, copy);
  }
  return (int)e;
}

// How many clusters of `cl` CTAs with `smem` bytes each can be resident at once.
template <class Ar>
int max_active_clusters(int cl, size_t smem) {
  auto kern = mgs_cluster_kernel<Ar, true>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cl);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = cl;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) return 0;
  return n;
}

int launch_d(const Params& pr, int grid, size_t smem, cudaStream_t stream, int kind);
int launch_cluster(int L, const Params& pr, int grid, int cl, size_t smem, cudaStream_t stream);
int cluster_capacity(int L, int cl, size_t smem);
int launch_dd(const Params& pr, int grid, size_t smem, cudaStream_t stream, int kind);
int launch_qd(const Params& pr, int grid, size_t smem, cudaStream_t stream, int kind);

}  // namespace mgs
