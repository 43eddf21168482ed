// C ABI of the batched least-squares solve: workspace layout, tuning parameters, launch.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/mgs_ddqd.h"
#include "batched_kernel.cuh"

namespace mgs {
void set_last_cuda_error(int code);
}

namespace {

struct BPlan {
  int T, per_sm, grid;
  size_t smem, off_scr, total;
  long long per_cta;
};

bool make_bplan(int L, int batch, int max_m, int max_n, const mgs_tune* tune, BPlan& bp) {
  if ((L != 2 && L != 4) || batch < 1 || max_n < 1 || max_m < max_n) return false;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
  bp.T = (tune && tune->threads) ? tune->threads : 128;
  bp.per_sm = (tune && tune->ctas_per_sm) ? tune->ctas_per_sm : 2;
  if (bp.T != 128 && bp.T != 256) return false;
  if (bp.per_sm < 1 || bp.per_sm > 4) return false;
  bp.smem = mgs::batched_smem_bytes(L, bp.T, max_m, max_n);
  if (bp.smem > 227 * 1024) return false;
  bp.grid = sms * bp.per_sm;
  if (bp.grid > batch) bp.grid = batch;
  bp.per_cta = mgs::batched_scratch_doubles(L, max_n);
  bp.off_scr = 256;
  bp.total = bp.off_scr + sizeof(double) * (size_t)bp.per_cta * bp.grid;
  return true;
}

template <class Ar, int T>
int launch_batched(const mgs::BatchParams& p, const BPlan& pl, cudaStream_t st) {
  auto kern = mgs::mgs_batched_kernel<Ar, T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
  if (e != cudaSuccess) return (int)e;
  mgs::BatchParams copy = p;
  void* args[] = {&copy};
  e = cudaLaunchKernel((const void*)kern, dim3(pl.grid), dim3(T), args, pl.smem, st);
  return (int)e;
}

int run_batched(int L, double* A, double* b, double* x, const int64_t* a_off, const int64_t* b_off,
                const int64_t* x_off, const int32_t* m_arr, const int32_t* n_arr, const int32_t* order, int batch,
                int max_m, int max_n, void* ws, size_t ws_bytes, int32_t* dev_status, const mgs_tune* tune,
                void* stream) {
  if (!A || !b || !x || !a_off || !b_off || !x_off || !m_arr || !n_arr || !ws || !dev_status) return MGS_EINVAL;
  if (batch < 1 || max_n < 1 || max_m < max_n) return MGS_EINVAL;
  auto mis = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; };
  if (mis(A) || mis(b) || mis(x) || mis(ws) || (reinterpret_cast<uintptr_t>(a_off) & 7u) ||
      (reinterpret_cast<uintptr_t>(b_off) & 7u) || (reinterpret_cast<uintptr_t>(x_off) & 7u) ||
      (reinterpret_cast<uintptr_t>(m_arr) & 3u) || (reinterpret_cast<uintptr_t>(n_arr) & 3u) ||
      (order && (reinterpret_cast<uintptr_t>(order) & 3u)) || (reinterpret_cast<uintptr_t>(dev_status) & 3u))
    return MGS_EINVAL;
  BPlan pl;
  if (!make_bplan(L, batch, max_m, max_n, tune, pl)) return MGS_ENOSPACE;
  if (ws_bytes < pl.total) return MGS_ENOSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* wb = static_cast<char*>(ws);
  cudaError_t e = cudaMemsetAsync(wb, 0, 256, st);
  if (e != cudaSuccess) {
    mgs::set_last_cuda_error((int)e);
    return MGS_ECUDA;
  }
  mgs::BatchParams p{};
  p.A = A;
  p.b = b;
  p.x = x;
  p.a_off = reinterpret_cast<const long long*>(a_off);
  p.b_off = reinterpret_cast<const long long*>(b_off);
  p.x_off = reinterpret_cast<const long long*>(x_off);
  p.m_arr = m_arr;
  p.n_arr = n_arr;
  p.order = order;
  p.batch = batch;
  p.max_m = max_m;
  p.max_n = max_n;
  p.counter = reinterpret_cast<unsigned*>(wb);
  p.ws = reinterpret_cast<double*>(wb + pl.off_scr);
  p.per_cta = pl.per_cta;
  p.status = dev_status;
  p.one = 1.0;
  p.nzero = -0.0;
  int rc;
  if (L == 2)
    rc = (pl.T == 128) ? launch_batched<mgs::DD, 128>(p, pl, st) : launch_batched<mgs::DD, 256>(p, pl, st);
  else
    rc = (pl.T == 128) ? launch_batched<mgs::QD, 128>(p, pl, st) : launch_batched<mgs::QD, 256>(p, pl, st);
  if (rc != 0) {
    mgs::set_last_cuda_error(rc);
    return MGS_ECUDA;
  }
  return MGS_OK;
}

}  // namespace

extern "C" {

size_t mgs_batched_workspace_bytes(int limbs, int batch, int max_m, int max_n, const mgs_tune* tune) {
  BPlan pl;
  if (!make_bplan(limbs, batch, max_m, max_n, tune, pl)) return 0;
  return pl.total;
}

int ls_solve_dd_batched(double* A_pool, double* b_pool, double* x_pool, const int64_t* a_off, const int64_t* b_off,
                        const int64_t* x_off, const int32_t* m, const int32_t* n, const int32_t* order, int batch,
                        int max_m, int max_n, void* workspace, size_t workspace_bytes, int32_t* dev_status,
                        const mgs_tune* tune, void* stream) {
  return run_batched(2, A_pool, b_pool, x_pool, a_off, b_off, x_off, m, n, order, batch, max_m, max_n, workspace,
                     workspace_bytes, dev_status, tune, stream);
}

int ls_solve_qd_batched(double* A_pool, double* b_pool, double* x_pool, const int64_t* a_off, const int64_t* b_off,
                        const int64_t* x_off, const int32_t* m, const int32_t* n, const int32_t* order, int batch,
                        int max_m, int max_n, void* workspace, size_t workspace_bytes, int32_t* dev_status,
                        const mgs_tune* tune, void* stream) {
  return run_batched(4, A_pool, b_pool, x_pool, a_off, b_off, x_off, m, n, order, batch, max_m, max_n, workspace,
                     workspace_bytes, dev_status, tune, stream);
}

}  // extern "C"
