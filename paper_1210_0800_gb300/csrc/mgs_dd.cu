// Complex double-double instantiation of the persistent MGS least-squares kernel.
#include "launch.cuh"

namespace mgs {
int launch_dd(const Params& pr, int grid, size_t smem, cudaStream_t stream, int kind) {
  return launch_kernel<DD>(pr, grid, smem, stream, kind);
}
int launch_cluster_dd(const Params& pr, int grid, int cl, size_t smem, cudaStream_t stream) {
  return launch_cluster_kernel<DD>(pr, grid, cl, smem, stream);
}
int cluster_capacity_dd(int cl, size_t smem) { return max_active_clusters<DD>(cl, smem); }
int blocks_per_sm_dd(int kind, size_t smem) { return blocks_per_sm<DD>(kind, smem); }
}  // namespace mgs
