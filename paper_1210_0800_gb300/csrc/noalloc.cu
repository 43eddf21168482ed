// ls_solve_dd_noalloc: the double-double least-squares solve for callers that cannot
// allocate device memory.  Some hosts own every device allocation themselves (a framework
// allocator, or an application that must not allocate once it has started), so a caller
// may have nowhere to get the workspace of ls_solve_dd from.  This entry point needs none:
// its scratch is a fixed array compiled into the library, and it calls no allocator.
//
// The array is a file-scope __device__ variable, so every GPU that loads the library
// holds MGS_NOALLOC_WORKSPACE_BYTES of it until the process exits.  Host code cannot use
// the variable's name as a device address, so the first call on each device looks the
// address up with cudaGetSymbolAddress (with that device current) and caches it; make
// that first call before any stream capture.  All calls share the array: calls whose
// execution may overlap on the GPU race on it and must not be issued.  Each call starts
// by clearing the parts that must start at zero (the solve's memsets), so the contents a
// previous call left behind do not matter.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/mgs_ddqd.h"

namespace mgs {
void set_last_cuda_error(int code);
}

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[MGS_NOALLOC_WORKSPACE_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" int ls_solve_dd_noalloc(double* A, int lda, double* b, double* x, double* R, int ldr, double* z, int m,
                                   int n, int32_t* dev_status, void* stream) {
  if (n < 1 || m < n || lda < m) return MGS_EINVAL;
  const size_t need = mgs_workspace_bytes(2, m, n, 1);
  if (need == 0 || need > (size_t)MGS_NOALLOC_WORKSPACE_BYTES) return MGS_ENOSPACE;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    mgs::set_last_cuda_error((int)e);
    return MGS_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return MGS_EINVAL;
  void* ws = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (g_scratch_addr[dev] == nullptr) {
      e = cudaGetSymbolAddress(&ws, g_noalloc_scratch);
      if (e != cudaSuccess) {
        mgs::set_last_cuda_error((int)e);
        return MGS_ECUDA;
      }
      g_scratch_addr[dev] = ws;
    }
    ws = g_scratch_addr[dev];
  }
  return ls_solve_dd(A, lda, b, x, R, ldr, z, m, n, ws, (size_t)MGS_NOALLOC_WORKSPACE_BYTES, dev_status, stream);
}
