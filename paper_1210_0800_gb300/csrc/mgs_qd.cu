// Complex quad-double instantiation of the persistent MGS least-squares kernel.
#include "launch.cuh"

namespace mgs {
int launch_qd(const Params& pr, int grid, size_t smem, cudaStream_t stream) {
  return launch_kernel<QD>(pr, grid, smem, stream);
}
}  // namespace mgs
