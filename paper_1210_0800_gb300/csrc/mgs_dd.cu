// Complex double-double instantiation of the persistent MGS least-squares kernel.
#include "launch.cuh"

namespace mgs {
int launch_dd(const Params& pr, int grid, size_t smem, cudaStream_t stream) {
  return launch_kernel<DD>(pr, grid, smem, stream);
}
}  // namespace mgs
