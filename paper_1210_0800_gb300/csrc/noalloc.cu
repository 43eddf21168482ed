// ls_solve_dd_noalloc: the double-double least-squares solve for callers that cannot
// allocate device memory.  Some hosts own every device allocation themselves (a framework
// allocator, or an application that must not allocate once it has started), so a caller
// may have nowhere to get the workspace of ls_solve_dd from.  This entry point needs none:
// its scratch is a fixed array compiled into the library, and it calls no allocator.
//
// The array is a file-scope __device__ variable.  Under lazy module loading (the CUDA
// default) the driver loads this file's module, and with it reserves the array's
// MGS_NOALLOC_WORKSPACE_BYTES on the device, at the first call on each device and
// context; the array then stays until the context is destroyed (normally at process exit).
// Host code cannot use the variable's name as a device address, so that first call looks
// the address up with cudaGetSymbolAddress (with the device current) and caches it per
// (device, context): a device reset or a new context gets a new module, possibly at
// another address, and a fresh lookup.  Make the first call at start-up, before the
// host's allocator takes the rest of device memory and before any stream capture.
// All calls share the array: calls whose execution may overlap on the GPU race on it and
// must not be issued.  Each call starts by clearing the parts that must start at zero
// (the solve's memsets), so the contents a previous call left behind do not matter.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/mgs_ddqd.h"

namespace mgs {
void set_last_cuda_error(int code);
}

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[MGS_NOALLOC_WORKSPACE_BYTES];

// The calling thread's current driver context, through the runtime's driver entry point
// (the library does not link the driver API); null when the lookup is not available.
using CtxGetCurrentFn = int (*)(void**);

CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (CtxGetCurrentFn) nullptr;
    return reinterpret_cast<CtxGetCurrentFn>(p);
  }();
  return fn;
}

struct Slot {
  int dev;
  void* ctx;
  void* addr;
};
constexpr int kSlots = 64;
std::mutex g_mutex;
Slot g_slots[kSlots];
int g_used = 0;

// Device address of the scratch array for the current device and context.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  void* ctx = nullptr;
  const CtxGetCurrentFn get = ctx_get_current();
  if (get == nullptr || get(&ctx) != 0 || ctx == nullptr) {
    // no context handle to key a cache on (or the runtime has not made the device's
    // context current yet; the lookup below does): look the address up this time
    return cudaGetSymbolAddress(out, g_noalloc_scratch);
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  for (int i = 0; i < g_used; ++i)
    if (g_slots[i].dev == dev && g_slots[i].ctx == ctx) {
      *out = g_slots[i].addr;
      return cudaSuccess;
    }
  void* addr = nullptr;
  e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  if (g_used < kSlots) {
    g_slots[g_used++] = Slot{dev, ctx, addr};
  } else {
    g_slots[(unsigned)dev % kSlots] = Slot{dev, ctx, addr};
  }
  *out = addr;
  return cudaSuccess;
}

}  // namespace

extern "C" int ls_solve_dd_noalloc(double* A, int lda, double* b, double* x, double* R, int ldr, double* z, int m,
                                   int n, int32_t* dev_status, void* stream) {
  if (n < 1 || m < n || lda < m) return MGS_EINVAL;
  const size_t need = mgs_workspace_bytes(2, m, n, 1);
  if (need == 0 || need > (size_t)MGS_NOALLOC_WORKSPACE_BYTES) return MGS_ENOSPACE;
  void* ws = nullptr;
  const cudaError_t e = scratch_address(&ws);
  if (e != cudaSuccess) {
    mgs::set_last_cuda_error((int)e);
    return MGS_ECUDA;
  }
  return ls_solve_dd(A, lda, b, x, R, ldr, z, m, n, ws, (size_t)MGS_NOALLOC_WORKSPACE_BYTES, dev_status, stream);
}
