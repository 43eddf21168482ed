// Complex double-double instantiation of the persistent MGS least-squares kernel.
#include "launch.cuh"

namespace mgs {
int launch_dd(const Params& pr, int grid, int T, size_t smem, cudaStream_t stream, int kind) {
  return launch_kernel<DD>(pr, grid, T, smem, stream, kind);
}
int launch_cluster_dd(const Params& pr, int grid, int cl, int T, size_t smem, cudaStream_t stream) {
  return launch_cluster_kernel<DD>(pr, grid, cl, T, smem, stream);
}
int cluster_capacity_dd(int cl, int T, size_t smem) { return max_active_clusters<DD>(cl, T, smem); }
int blocks_per_sm_dd(int kind, int T, size_t smem) { return blocks_per_sm<DD>(kind, T, smem); }
}  // namespace mgs
