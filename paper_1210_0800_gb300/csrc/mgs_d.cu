// Complex double (one FP64 limb) instantiation of the persistent MGS least-squares kernel.
#include "launch.cuh"

namespace mgs {
int launch_d(const Params& pr, int grid, int T, size_t smem, cudaStream_t stream, int kind) {
  return launch_kernel<D>(pr, grid, T, smem, stream, kind);
}
int launch_cluster_d(const Params& pr, int grid, int cl, int T, size_t smem, cudaStream_t stream) {
  return launch_cluster_kernel<D>(pr, grid, cl, T, smem, stream);
}
int cluster_capacity_d(int cl, int T, size_t smem) { return max_active_clusters<D>(cl, T, smem); }
int blocks_per_sm_d(int kind, int T, size_t smem) { return blocks_per_sm<D>(kind, T, smem); }
}  // namespace mgs
