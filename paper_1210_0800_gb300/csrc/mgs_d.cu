// Complex double (one FP64 limb) instantiation of the persistent MGS least-squares kernel.
#include "launch.cuh"

namespace mgs {
int launch_d(const Params& pr, int grid, size_t smem, cudaStream_t stream) {
  return launch_kernel<D>(pr, grid, smem, stream);
}
}  // namespace mgs
