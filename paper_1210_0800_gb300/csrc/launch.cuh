// Launch of the persistent single-system MGS kernels.  All CTAs must be co-resident (the
// kernels' barriers and pivot flags rely on it): the plan checks residency once per
// layout (blocks_per_sm, max_active_clusters), the launches are cooperative where the
// driver allows it, and every wait in the kernels is bounded.
#pragma once

#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "mgs_cluster.cuh"
#include "mgs_kernel.cuh"

namespace mgs {

// Raises a kernel's dynamic shared-memory limit on the current device once (again only
// when more is asked for), so that a launch costs no attribute call.
inline cudaError_t ensure_smem(const void* kern, size_t smem) {
  struct Entry {
    const void* kern;
    int dev;
    size_t bytes;
  };
  static std::mutex mu;
  static std::vector<Entry> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> g(mu);
  for (Entry& d : done)
    if (d.kern == kern && d.dev == dev) {
      if (d.bytes >= smem) return cudaSuccess;
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) d.bytes = smem;
      return e;
    }
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) done.push_back(Entry{kern, dev, smem});
  return e;
}

// kind 0: mgs_ls_kernel (a grid barrier per step); kind 2: the cluster schedule with
// software groups (mgs_cluster_kernel<Ar, false>); T threads per CTA (128 or 256).
template <class Ar>
const void* grid_kernel(int kind, int T) {
  if (T == 256) return kind == 2 ? (const void*)mgs_cluster_kernel<Ar, false, 256> : (const void*)mgs_ls_kernel<Ar, 256>;
  return kind == 2 ? (const void*)mgs_cluster_kernel<Ar, false, 128> : (const void*)mgs_ls_kernel<Ar, 128>;
}
template <class Ar>
const void* cluster_kernel(int T) {
  return T == 256 ? (const void*)mgs_cluster_kernel<Ar, true, 256> : (const void*)mgs_cluster_kernel<Ar, true, 128>;
}

// Resident CTAs per SM of a plain-grid kernel with `smem` bytes of shared memory.
template <class Ar>
int blocks_per_sm(int kind, int T, size_t smem) {
  const void* kern = grid_kernel<Ar>(kind, T);
  if (ensure_smem(kern, smem) != cudaSuccess) return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T, smem) != cudaSuccess) return 0;
  return per_sm;
}

template <class Ar>
int launch_kernel(const Params& pr, int grid, int T, size_t smem, cudaStream_t stream, int kind) {
  const void* kern = grid_kernel<Ar>(kind, T);
  cudaError_t e = ensure_smem(kern, smem);
  if (e != cudaSuccess) return (int)e;
  Params copy = pr;
  void* args[] = {&copy};
  return (int)cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(T), args, smem, stream);
}

// Cluster variant: clusters of `cl` CTAs (the row blocks of a column group).  Launched
// cooperatively when the driver accepts cooperative cluster launches, otherwise as a plain
// cluster launch (the plan has checked that every cluster can be resident at once).
template <class Ar>
int launch_cluster_kernel(const Params& pr, int grid, int cl, int T, size_t smem, cudaStream_t stream) {
  const void* kern = cluster_kernel<Ar>(T);
  cudaError_t e = ensure_smem(kern, smem);
  if (e != cudaSuccess) return (int)e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(T);
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
  Params copy = pr;
  void* args[] = {&copy};
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(stream, &cap);
  if (e != cudaSuccess) return (int)e;
  if (cap != cudaStreamCaptureStatusNone) {
    // inside a capture a refused launch would invalidate the graph: no second try
    cfg.numAttrs = 1;
    return (int)cudaLaunchKernelExC(&cfg, kern, args);
  }
  cfg.numAttrs = 2;
  e = cudaLaunchKernelExC(&cfg, kern, args);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    cfg.numAttrs = 1;
    e = cudaLaunchKernelExC(&cfg, kern, args);
  }
  return (int)e;
}

// How many clusters of `cl` CTAs with `smem` bytes each can be resident at once.
template <class Ar>
int max_active_clusters(int cl, int T, size_t smem) {
  const void* kern = cluster_kernel<Ar>(T);
  if (ensure_smem(kern, smem) != cudaSuccess) return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cl);
  cfg.blockDim = dim3(T);
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

int launch_d(const Params& pr, int grid, int T, size_t smem, cudaStream_t stream, int kind);
int launch_dd(const Params& pr, int grid, int T, size_t smem, cudaStream_t stream, int kind);
int launch_qd(const Params& pr, int grid, int T, size_t smem, cudaStream_t stream, int kind);
int launch_cluster(int L, const Params& pr, int grid, int cl, int T, size_t smem, cudaStream_t stream);
int cluster_capacity(int L, int cl, int T, size_t smem);
int grid_capacity(int L, int kind, int T, size_t smem);

}  // namespace mgs
