// C ABI of the MGS least-squares library: argument checks, the Br x Bc decomposition,
// the workspace layout and the launch.  See include/mgs_ddqd.h for the contract.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>

#include "../../include/mgs_ddqd.h"
#include "launch.cuh"

namespace {

thread_local int g_last_cuda = 0;

constexpr int kMaxBr = 32;             // partial reduction uses one warp-shuffle group
constexpr size_t kMaxSmem = 227 * 1024;  // dynamic shared memory per CTA on sm_103a
constexpr long long kTimeoutNs = 4000000000LL;  // 4 s: far above any legitimate wait

struct Plan {
  int L, m, n, nc, aug;
  int Br, Bc, h, w;
  size_t smem;
  size_t off_sync, off_flags, off_P, off_V, off_Y, off_R, off_G, off_T, total, zero_bytes;
};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return sms;
}

// Rows per CTA about 64; as many column groups as SMs allow; every row block non-empty.
bool make_plan(int L, int m, int n, int aug, Plan& pl) {
  if ((L != 1 && L != 2 && L != 4) || n < 1 || m < n) return false;
  const int sms = device_sms();
  if (sms <= 0) return false;
  pl.L = L;
  pl.m = m;
  pl.n = n;
  pl.aug = aug ? 1 : 0;
  pl.nc = n + pl.aug;
  const int E = 2 * L;
  int h = 64;
  for (;;) {
    int Br = (m + h - 1) / h;
    if (Br > kMaxBr || Br > sms) return false;
    int Bc = sms / Br;
    if (Bc > pl.nc) Bc = pl.nc;
    if (Bc < 1) return false;
    const int w = (pl.nc + Bc - 1) / Bc;
    size_t smem = mgs::smem_bytes(L, h, w);
    const size_t bs = sizeof(double) * ((size_t)(mgs::kBS + 1) * E) + 64;  // back substitution
    if (bs > smem) smem = bs;
    if (smem <= kMaxSmem) {
      pl.Br = Br;
      pl.Bc = Bc;
      pl.h = h;
      pl.w = w;
      pl.smem = smem;
      break;
    }
    if (h <= 8) return false;
    h /= 2;
  }
  size_t off = 0;
  pl.off_sync = off;
  off = align256(off + 64);
  pl.off_flags = off;
  off = align256(off + sizeof(int) * (size_t)(pl.nc + 1) * pl.Br);
  pl.zero_bytes = off;
  const int ACC = (L == 1) ? mgs::D::ACC : (L == 2) ? mgs::DD::ACC : mgs::QD::ACC;
  pl.off_P = off;
  off = align256(off + sizeof(double) * 2 * (size_t)pl.Br * pl.nc * ACC);
  pl.off_V = off;
  off = align256(off + sizeof(double) * 2 * (size_t)pl.Br * pl.h * E);
  pl.off_Y = off;
  off = align256(off + sizeof(double) * (size_t)pl.nc * E);
  pl.off_R = off;
  off = align256(off + sizeof(double) * (size_t)n * n * E);
  pl.off_G = off;  // G_kk, r_kk, 1/r_kk
  off = align256(off + sizeof(double) * 3 * (size_t)pl.nc * L);
  pl.off_T = off;
#if defined(MGS_TRACE) && MGS_TRACE
  off = align256(off + sizeof(unsigned long long) * 8 * (size_t)(pl.nc + 1) * pl.Br * pl.Bc);
#endif
  pl.total = off;
  return true;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int run(int L, double* A, int lda, double* b, double* x, double* R, int ldr, double* z, int m, int n, void* ws,
        size_t ws_bytes, int32_t* dev_status, void* stream, int aug) {
  if (!A || !dev_status || !ws) return MGS_EINVAL;
  if (aug && (!b || !x)) return MGS_EINVAL;
  if (!aug && !R) return MGS_EINVAL;
  if (n < 1 || m < n || lda < m) return MGS_EINVAL;
  if (R && ldr < n) return MGS_EINVAL;
  if (!aligned16(A) || (b && !aligned16(b)) || (x && !aligned16(x)) || (R && !aligned16(R)) ||
      (z && !aligned16(z)) || !aligned16(ws) || (reinterpret_cast<uintptr_t>(dev_status) & 3u))
    return MGS_EINVAL;
  Plan pl;
  if (!make_plan(L, m, n, aug, pl)) return MGS_ENOSPACE;
  if (ws_bytes < pl.total) return MGS_ENOSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* wb = static_cast<char*>(ws);
  cudaError_t e = cudaMemsetAsync(wb, 0, pl.zero_bytes, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dev_status, 0, sizeof(int32_t), st);
  if (e != cudaSuccess) {
    g_last_cuda = (int)e;
    return MGS_ECUDA;
  }
  mgs::Params pr{};
  pr.A = A;
  pr.lda = lda;
  pr.b = aug ? b : nullptr;
  pr.R = R ? R : reinterpret_cast<double*>(wb + pl.off_R);
  pr.ldr = R ? ldr : n;
  pr.Rt = reinterpret_cast<double*>(wb + pl.off_R);
  pr.x = aug ? x : nullptr;
  pr.z = aug ? z : nullptr;
  pr.m = m;
  pr.n = n;
  pr.nc = pl.nc;
  pr.aug = pl.aug;
  pr.Br = pl.Br;
  pr.Bc = pl.Bc;
  pr.h = pl.h;
  pr.sync = reinterpret_cast<unsigned*>(wb + pl.off_sync);
  pr.flags = reinterpret_cast<int*>(wb + pl.off_flags);
  pr.P = reinterpret_cast<double*>(wb + pl.off_P);
  pr.V = reinterpret_cast<double*>(wb + pl.off_V);
  pr.Y = reinterpret_cast<double*>(wb + pl.off_Y);
  pr.Gd = reinterpret_cast<double*>(wb + pl.off_G);
  pr.Rd = pr.Gd + (size_t)pl.nc * L;
  pr.Ri = pr.Rd + (size_t)pl.nc * L;
  pr.status = dev_status;
  pr.one = 1.0;
  pr.nzero = -0.0;
  pr.timeout_ns = kTimeoutNs;
#if defined(MGS_TRACE) && MGS_TRACE
  pr.trace = reinterpret_cast<unsigned long long*>(wb + pl.off_T);
#else
  pr.trace = nullptr;
#endif
  const int grid = pl.Br * pl.Bc;
  const int rc = (L == 1)   ? mgs::launch_d(pr, grid, pl.smem, st)
                 : (L == 2) ? mgs::launch_dd(pr, grid, pl.smem, st)
                            : mgs::launch_qd(pr, grid, pl.smem, st);
  if (rc != 0) {
    g_last_cuda = rc;
    return MGS_ECUDA;
  }
  return MGS_OK;
}

}  // namespace

namespace mgs {
// Lets the other translation units of the library record a CUDA error for
// mgs_last_cuda_error().
void set_last_cuda_error(int code) { g_last_cuda = code; }
}  // namespace mgs

extern "C" {

int mgs_version(void) { return 100; }

const char* mgs_status_string(int code) {
  switch (code) {
    case MGS_OK: return "MGS_OK";
    case MGS_EINVAL: return "MGS_EINVAL";
    case MGS_ERANK: return "MGS_ERANK";
    case MGS_ENONFINITE: return "MGS_ENONFINITE";
    case MGS_ETIMEOUT: return "MGS_ETIMEOUT";
    case MGS_ECUDA: return "MGS_ECUDA";
    case MGS_ENOSPACE: return "MGS_ENOSPACE";
    default: return "MGS_UNKNOWN";
  }
}

int mgs_last_cuda_error(void) { return g_last_cuda; }

#if defined(MGS_TRACE) && MGS_TRACE
// Trace builds only: where the phase timestamps sit in the workspace.
__attribute__((visibility("default"))) int mgs_trace_layout(int limbs, int m, int n, int with_rhs,
                                                            size_t* offset, int* steps, int* ctas) {
  Plan pl;
  if (!make_plan(limbs, m, n, with_rhs, pl)) return MGS_ENOSPACE;
  *offset = pl.off_T;
  *steps = pl.nc + 1;
  *ctas = pl.Br * pl.Bc;
  return MGS_OK;
}
#endif

size_t mgs_workspace_bytes(int limbs, int m, int n, int with_rhs) {
  Plan pl;
  if (!make_plan(limbs, m, n, with_rhs, pl)) return 0;
  return pl.total;
}

int mgs_qr_d(double* A, int lda, double* R, int ldr, int m, int n, void* workspace, size_t workspace_bytes,
             int32_t* dev_status, void* stream) {
  return run(1, A, lda, nullptr, nullptr, R, ldr, nullptr, m, n, workspace, workspace_bytes, dev_status, stream, 0);
}

int ls_solve_d(double* A, int lda, double* b, double* x, double* R, int ldr, double* z, int m, int n, void* workspace,
               size_t workspace_bytes, int32_t* dev_status, void* stream) {
  return run(1, A, lda, b, x, R, ldr, z, m, n, workspace, workspace_bytes, dev_status, stream, 1);
}

int mgs_qr_dd(double* A, int lda, double* R, int ldr, int m, int n, void* workspace, size_t workspace_bytes,
              int32_t* dev_status, void* stream) {
  return run(2, A, lda, nullptr, nullptr, R, ldr, nullptr, m, n, workspace, workspace_bytes, dev_status, stream, 0);
}

int mgs_qr_qd(double* A, int lda, double* R, int ldr, int m, int n, void* workspace, size_t workspace_bytes,
              int32_t* dev_status, void* stream) {
  return run(4, A, lda, nullptr, nullptr, R, ldr, nullptr, m, n, workspace, workspace_bytes, dev_status, stream, 0);
}

int ls_solve_dd(double* A, int lda, double* b, double* x, double* R, int ldr, double* z, int m, int n,
                void* workspace, size_t workspace_bytes, int32_t* dev_status, void* stream) {
  return run(2, A, lda, b, x, R, ldr, z, m, n, workspace, workspace_bytes, dev_status, stream, 1);
}

int ls_solve_qd(double* A, int lda, double* b, double* x, double* R, int ldr, double* z, int m, int n,
                void* workspace, size_t workspace_bytes, int32_t* dev_status, void* stream) {
  return run(4, A, lda, b, x, R, ldr, z, m, n, workspace, workspace_bytes, dev_status, stream, 1);
}

}  // extern "C"
