// Complex quad-double instantiation of the persistent MGS least-squares kernel.
#include "launch.cuh"

namespace mgs {
int launch_qd(const Params& pr, int grid, int T, size_t smem, cudaStream_t stream, int kind) {
  return launch_kernel<QD>(pr, grid, T, smem, stream, kind);
}
int launch_cluster_qd(const Params& pr, int grid, int cl, int T, size_t smem, cudaStream_t stream) {
  return launch_cluster_kernel<QD>(pr, grid, cl, T, smem, stream);
}
int cluster_capacity_qd(int cl, int T, size_t smem) { return max_active_clusters<QD>(cl, T, smem); }
int blocks_per_sm_qd(int kind, int T, size_t smem) { return blocks_per_sm<QD>(kind, T, smem); }
}  // namespace mgs
