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
  int T, per_sm, grid, S;  // S: CTAs per system (a thread-block cluster when > 1)
  int cmax;                // lanes per (column, part) cap (0 = none)
  size_t smem, off_scr, total;
  long long per_cta;
};

bool make_bplan(int L, int batch, int max_m, int max_n, const mgs_tune* tune, BPlan& bp) {
  if ((L != 1 && L != 2 && L != 4) || batch < 1 || max_n < 1 || max_m < max_n) return false;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
  bp.T = (tune && tune->threads) ? tune->threads : 256;
  bp.per_sm = (tune && tune->ctas_per_sm) ? tune->ctas_per_sm : 1;
  if (bp.T != 128 && bp.T != 256) return false;
  if (bp.per_sm < 1 || bp.per_sm > 4) return false;
  bp.cmax = tune ? tune->chunks : 0;
  if (bp.cmax < 0 || bp.cmax > bp.T) return false;
  // systems split over S CTAs when the batch is smaller than the GPU (each slice keeps at
  // least 32 rows); automatic unless the tuning asks for a split
  if (tune && tune->split) {
    bp.S = tune->split;
    if (bp.S != 1 && bp.S != 2 && bp.S != 4) return false;
  } else {
    bp.S = 1;
    while (bp.S < 4 && (long long)batch * 2 * bp.S <= (long long)sms * bp.per_sm && max_m / (2 * bp.S) >= 32)
      bp.S *= 2;
  }
  bp.smem = mgs::batched_smem_bytes(L, bp.T, max_m, max_n, bp.S);
  if (bp.smem > 227 * 1024) return false;
  const int clusters = (sms * bp.per_sm) / bp.S;
  bp.grid = bp.S * (clusters < batch ? clusters : batch);
  bp.per_cta = mgs::batched_scratch_doubles(L, max_n);
  bp.off_scr = 256;
  bp.total = bp.off_scr + sizeof(double) * (size_t)bp.per_cta * bp.grid;
  return true;
}

template <class Ar, int T, int S>
int launch_batched_s(const mgs::BatchParams& p, const BPlan& pl, cudaStream_t st) {
  auto kern = mgs::mgs_batched_kernel<Ar, T, S>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
  if (e != cudaSuccess) return (int)e;
  mgs::BatchParams copy = p;
  void* args[] = {&copy};
  if constexpr (S == 1) {
    return (int)cudaLaunchKernel((const void*)kern, dim3(pl.grid), dim3(T), args, pl.smem, st);
  } else {
    // the clusters work independently (no CTA waits for another cluster)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(pl.grid);
    cfg.blockDim = dim3(T);
    cfg.dynamicSmemBytes = pl.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = S;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return (int)cudaLaunchKernelExC(&cfg, (const void*)kern, args);
  }
}

template <class Ar, int T>
int launch_batched(const mgs::BatchParams& p, const BPlan& pl, cudaStream_t st) {
  return pl.S == 4 ? launch_batched_s<Ar, T, 4>(p, pl, st)
         : pl.S == 2 ? launch_batched_s<Ar, T, 2>(p, pl, st)
                     : launch_batched_s<Ar, T, 1>(p, pl, st);
}

int run_batched(int L, double* A, double* b, double* x, double* R, const int64_t* a_off, const int64_t* b_off,
                const int64_t* x_off, const int64_t* r_off, const int32_t* m_arr, const int32_t* n_arr,
                const int32_t* order, int batch, int max_m, int max_n, void* ws, size_t ws_bytes, int32_t* dev_status,
                const mgs_tune* tune, void* stream) {
  if (!A || !b || !x || !a_off || !b_off || !x_off || !m_arr || !n_arr || !ws || !dev_status) return MGS_EINVAL;
  if (R && (!r_off || (reinterpret_cast<uintptr_t>(R) & 15u) || (reinterpret_cast<uintptr_t>(r_off) & 7u)))
    return MGS_EINVAL;
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
  p.R = R;
  p.r_off = reinterpret_cast<const long long*>(r_off);
  p.batch = batch;
  p.max_m = max_m;
  p.max_n = max_n;
  p.counter = reinterpret_cast<unsigned*>(wb);
  p.ws = reinterpret_cast<double*>(wb + pl.off_scr);
  p.per_cta = pl.per_cta;
  p.status = dev_status;
  p.cmax = pl.cmax;
  p.one = 1.0;
  p.nzero = -0.0;
  int rc;
  if (L == 1)
    rc = (pl.T == 128) ? launch_batched<mgs::D, 128>(p, pl, st) : launch_batched<mgs::D, 256>(p, pl, st);
  else if (L == 2)
    rc = (pl.T == 128) ? launch_batched<mgs::DD, 128>(p, pl, st) : launch_batched<mgs::DD, 256>(p, pl, st);
  else
    rc = (pl.T == 128) ? launch_batched<mgs::QD, 128>(p, pl, st) : launch_batched<mgs::QD, 256>(p, pl, st);
  if (rc != 0) {
    mgs::set_last_cuda_error(rc);
    return MGS_ECUDA;
  }
  return MGS_OK;
}

template <class Ar, int T>
int launch_adjoint(const mgs::AdjParams& p, int grid, size_t smem, cudaStream_t st) {
  auto kern = mgs::mgs_adjoint_kernel<Ar, T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  mgs::AdjParams copy = p;
  void* args[] = {&copy};
  return (int)cudaLaunchKernel((const void*)kern, dim3(grid), dim3(T), args, smem, st);
}

int run_adjoint(int L, const double* Q, const double* R, const double* x, const double* r, const double* G, double* gA,
                double* gb, const int64_t* a_off, const int64_t* r_off, const int64_t* b_off, const int64_t* x_off,
                const int32_t* m_arr, const int32_t* n_arr, const int32_t* order, int batch, int max_m, int max_n,
                void* ws, size_t ws_bytes, int32_t* dev_status, const mgs_tune* tune, void* stream) {
  if (!Q || !R || !x || !r || !G || !gA || !gb || !a_off || !r_off || !b_off || !x_off || !m_arr || !n_arr || !ws ||
      !dev_status)
    return MGS_EINVAL;
  if (batch < 1 || max_n < 1 || max_m < max_n) return MGS_EINVAL;
  auto mis = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; };
  if (mis(Q) || mis(R) || mis(x) || mis(r) || mis(G) || mis(gA) || mis(gb) || mis(ws)) return MGS_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))
    return MGS_ECUDA;
  const int T = (tune && tune->threads) ? tune->threads : 256;
  const int per_sm = (tune && tune->ctas_per_sm) ? tune->ctas_per_sm : 1;
  if ((T != 128 && T != 256) || per_sm < 1 || per_sm > 4) return MGS_EINVAL;
  const size_t smem = mgs::adjoint_smem_bytes(L, max_n);
  if (smem > 227 * 1024) return MGS_ENOSPACE;
  if (ws_bytes < 256) return MGS_ENOSPACE;
  int grid = sms * per_sm;
  if (grid > batch) grid = batch;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(ws, 0, 256, st);
  if (e != cudaSuccess) {
    mgs::set_last_cuda_error((int)e);
    return MGS_ECUDA;
  }
  mgs::AdjParams p{};
  p.Q = Q;
  p.R = R;
  p.x = x;
  p.r = r;
  p.G = G;
  p.gA = gA;
  p.gb = gb;
  p.a_off = reinterpret_cast<const long long*>(a_off);
  p.r_off = reinterpret_cast<const long long*>(r_off);
  p.b_off = reinterpret_cast<const long long*>(b_off);
  p.x_off = reinterpret_cast<const long long*>(x_off);
  p.m_arr = m_arr;
  p.n_arr = n_arr;
  p.order = order;
  p.batch = batch;
  p.max_m = max_m;
  p.max_n = max_n;
  p.counter = static_cast<unsigned*>(ws);
  p.status = dev_status;
  p.one = 1.0;
  p.nzero = -0.0;
  int rc;
  if (L == 2)
    rc = (T == 128) ? launch_adjoint<mgs::DD, 128>(p, grid, smem, st) : launch_adjoint<mgs::DD, 256>(p, grid, smem, st);
  else
    rc = (T == 128) ? launch_adjoint<mgs::QD, 128>(p, grid, smem, st) : launch_adjoint<mgs::QD, 256>(p, grid, smem, st);
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

int ls_solve_d_batched(double* A_pool, double* b_pool, double* x_pool, double* R_pool, const int64_t* a_off,
                       const int64_t* b_off, const int64_t* x_off, const int64_t* r_off, const int32_t* m,
                       const int32_t* n, const int32_t* order, int batch, int max_m, int max_n, void* workspace,
                       size_t workspace_bytes, int32_t* dev_status, const mgs_tune* tune, void* stream) {
  return run_batched(1, A_pool, b_pool, x_pool, R_pool, a_off, b_off, x_off, r_off, m, n, order, batch, max_m, max_n,
                     workspace, workspace_bytes, dev_status, tune, stream);
}

int ls_solve_dd_batched(double* A_pool, double* b_pool, double* x_pool, double* R_pool, const int64_t* a_off,
                        const int64_t* b_off, const int64_t* x_off, const int64_t* r_off, const int32_t* m,
                        const int32_t* n, const int32_t* order, int batch, int max_m, int max_n, void* workspace,
                        size_t workspace_bytes, int32_t* dev_status, const mgs_tune* tune, void* stream) {
  return run_batched(2, A_pool, b_pool, x_pool, R_pool, a_off, b_off, x_off, r_off, m, n, order, batch, max_m, max_n,
                     workspace, workspace_bytes, dev_status, tune, stream);
}

int ls_solve_qd_batched(double* A_pool, double* b_pool, double* x_pool, double* R_pool, const int64_t* a_off,
                        const int64_t* b_off, const int64_t* x_off, const int64_t* r_off, const int32_t* m,
                        const int32_t* n, const int32_t* order, int batch, int max_m, int max_n, void* workspace,
                        size_t workspace_bytes, int32_t* dev_status, const mgs_tune* tune, void* stream) {
  return run_batched(4, A_pool, b_pool, x_pool, R_pool, a_off, b_off, x_off, r_off, m, n, order, batch, max_m, max_n,
                     workspace, workspace_bytes, dev_status, tune, stream);
}

int ls_adjoint_dd_batched(const double* Q_pool, const double* R_pool, const double* x_pool, const double* r_pool,
                          const double* G_pool, double* gA_pool, double* gb_pool, const int64_t* a_off,
                          const int64_t* r_off, const int64_t* b_off, const int64_t* x_off, const int32_t* m,
                          const int32_t* n, const int32_t* order, int batch, int max_m, int max_n, void* workspace,
                          size_t workspace_bytes, int32_t* dev_status, const mgs_tune* tune, void* stream) {
  return run_adjoint(2, Q_pool, R_pool, x_pool, r_pool, G_pool, gA_pool, gb_pool, a_off, r_off, b_off, x_off, m, n,
                     order, batch, max_m, max_n, workspace, workspace_bytes, dev_status, tune, stream);
}

int ls_adjoint_qd_batched(const double* Q_pool, const double* R_pool, const double* x_pool, const double* r_pool,
                          const double* G_pool, double* gA_pool, double* gb_pool, const int64_t* a_off,
                          const int64_t* r_off, const int64_t* b_off, const int64_t* x_off, const int32_t* m,
                          const int32_t* n, const int32_t* order, int batch, int max_m, int max_n, void* workspace,
                          size_t workspace_bytes, int32_t* dev_status, const mgs_tune* tune, void* stream) {
  return run_adjoint(4, Q_pool, R_pool, x_pool, r_pool, G_pool, gA_pool, gb_pool, a_off, r_off, b_off, x_off, m, n,
                     order, batch, max_m, max_n, workspace, workspace_bytes, dev_status, tune, stream);
}

}  // extern "C"
