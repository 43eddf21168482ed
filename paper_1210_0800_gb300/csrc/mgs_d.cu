// Complex double (one FP64 limb) instantiation of the persistent MGS least-squares kernel.
#include "launch.cuh"

namespace mgs {
int launch_d(const Params& pr, int grid, size_t smem, cudaStream_t stream, int kind) {
  return launch_kernel<D>(pr, grid, smem, stream, kind);
}
int launch_cluster_d(const Params& pr, int grid, int cl, size_t smem, cudaStream_t stream) {
  return launch_cluster_kernel<D>(pr, grid, cl, smem, stream);
}
int cluster_capacity_d(int cl, size_t smem) { return max_active_clusters<D>(cl, smem); }
int blocks_per_sm_d(int kind, size_t smem) { return blocks_per_sm<D>(kind, smem); }
}  // namespace mgs
