// Newton corrector step on the device: the least-squares solve of the linearised system
// followed by the update of x, gated by a device-side state so that a whole corrector
// run can be enqueued (or captured in a CUDA graph) without a host synchronisation.
// Newton's method as the corrector of path tracking: the Jacobian and the system stay on
// the GPU and only the solutions go back to the host (Section 7); the Jacobian and the
// residual are the caller's.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/mgs_ddqd.h"
#include "mgs_kernel.cuh"

namespace mgs {
void set_last_cuda_error(int code);
int ls_solve_gated(int L, double* A, int lda, double* b, double* x, double* z, int m, int n, void* ws,
                   size_t ws_bytes, int32_t* dev_status, void* stream, const int32_t* skip);
}  // namespace mgs

namespace {

using mgs::Fp;
using mgs::g_load;
constexpr int kNT = 256;

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// |v| of a complex element from its leading limbs (a magnitude for the convergence test).
template <class Ar>
__device__ __forceinline__ double lead_abs(const double* e) {
  return hypot(e[0], e[Ar::L]);
}

__device__ __forceinline__ double block_max(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (kNT >> 5) ? red[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  }
  return v;  // valid in thread 0
}

// Before the solve: ||F(x_i)||_inf of the caller's residual (the right-hand side).
template <class Ar>
__global__ void __launch_bounds__(kNT) newton_pre_kernel(const double* F, int m, mgs_newton_state* st) {
  __shared__ double red[kNT / 32];
  if (st->done) return;
  constexpr int E = 2 * Ar::L;
  double v = 0.0;
  for (int i = threadIdx.x; i < m; i += kNT) v = fmax(v, lead_abs<Ar>(F + (size_t)i * E));
  v = block_max(v, red);
  const int it = st->iterations;
  if (threadIdx.x == 0 && it < MGS_NEWTON_HISTORY) st->f_norm[it] = v;
}

// After the solve of min ||F - J s||: x <- x - s (the Newton step dx = -s), the norms of
// the step and of x, the linearised residual z, and the stopping test
// ||dx||_inf <= tol ||x||_inf.  A solve that reported an error ends the run.
template <class Ar>
__global__ void __launch_bounds__(kNT) newton_update_kernel(double* x, const double* s, const double* z, int n,
                                                            double tol, const int32_t* solve_status,
                                                            mgs_newton_state* st, double one, double nzero) {
  __shared__ double red[kNT / 32];
  __shared__ int stop;
  if (st->done) return;
  constexpr int L = Ar::L, E = 2 * L;
  using elem = typename Ar::elem;
  const Fp f{one, nzero};
  if (threadIdx.x == 0) stop = *solve_status;
  __syncthreads();
  if (stop != 0) {
    if (threadIdx.x == 0) {
      st->done = 2;
      st->status = stop;
    }
    return;
  }
  elem c1;
#pragma unroll
  for (int q = 0; q < E; ++q) c1.v[q] = 0.0;
  c1.v[0] = 1.0;
  double dx = 0.0, xn = 0.0;
  for (int t = threadIdx.x; t < 2 * n; t += kNT) {
    const int j = t >> 1, part = t & 1;
    double* xj = x + (size_t)j * E;
    const elem sv = g_load<Ar>(s + (size_t)j * E);
    elem y = g_load<Ar>(xj);
    Ar::update_part(f, y, c1, sv, part);  // x_j - 1 * s_j, one part per lane
#pragma unroll
    for (int q = 0; q < L; ++q) xj[part * L + q] = y.v[part * L + q];
    if (part == 0) dx = fmax(dx, lead_abs<Ar>(s + (size_t)j * E));
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += kNT) xn = fmax(xn, lead_abs<Ar>(x + (size_t)j * E));
  dx = block_max(dx, red);
  __syncthreads();
  xn = block_max(xn, red);
  if (threadIdx.x == 0) {
    const int it = st->iterations;
    if (it < MGS_NEWTON_HISTORY) {
      st->dx_norm[it] = dx;
      st->x_norm[it] = xn;
      st->z[it] = z ? z[0] : 0.0;
    }
    st->iterations = it + 1;
    if (dx <= tol * xn) st->done = 1;
  }
}

template <class Ar>
int newton_step(double* J, int ldj, double* F, double* x, int m, int n, double tol, mgs_newton_state* st,
                void* ws, size_t ws_bytes, int32_t* dev_status, void* stream) {
  constexpr int L = Ar::L, E = 2 * L;
  if (!J || !F || !x || !st || !ws || !dev_status) return MGS_EINVAL;
  if (n < 1 || m < n || ldj < m || !(tol >= 0.0)) return MGS_EINVAL;
  if ((reinterpret_cast<uintptr_t>(x) & 15u) || (reinterpret_cast<uintptr_t>(st) & 15u)) return MGS_EINVAL;
  const size_t need = newton_workspace_bytes(L, m, n);
  if (need == 0 || ws_bytes < need) return MGS_ENOSPACE;
  const size_t solve_bytes = mgs_workspace_bytes(L, m, n, 1);
  char* wb = static_cast<char*>(ws);
  double* s = reinterpret_cast<double*>(wb + align256(solve_bytes));
  double* z = reinterpret_cast<double*>(wb + align256(solve_bytes) + align256(sizeof(double) * (size_t)n * E));
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  newton_pre_kernel<Ar><<<1, kNT, 0, cs>>>(F, m, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    mgs::set_last_cuda_error((int)e);
    return MGS_ECUDA;
  }
  const int rc = mgs::ls_solve_gated(L, J, ldj, F, s, z, m, n, ws, solve_bytes, dev_status, stream, &st->done);
  if (rc != MGS_OK) return rc;
  newton_update_kernel<Ar><<<1, kNT, 0, cs>>>(x, s, z, n, tol, dev_status, st, 1.0, -0.0);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    mgs::set_last_cuda_error((int)e);
    return MGS_ECUDA;
  }
  return MGS_OK;
}

}  // namespace

extern "C" {

size_t newton_workspace_bytes(int limbs, int m, int n) {
  const size_t sb = mgs_workspace_bytes(limbs, m, n, 1);
  if (sb == 0) return 0;
  return align256(sb) + align256(sizeof(double) * (size_t)n * 2 * limbs) + align256(sizeof(double) * limbs);
}

int newton_step_d(double* J, int ldj, double* F, double* x, int m, int n, double tol, mgs_newton_state* dev_state,
                  void* workspace, size_t workspace_bytes, int32_t* dev_status, void* stream) {
  return newton_step<mgs::D>(J, ldj, F, x, m, n, tol, dev_state, workspace, workspace_bytes, dev_status, stream);
}
int newton_step_dd(double* J, int ldj, double* F, double* x, int m, int n, double tol, mgs_newton_state* dev_state,
                   void* workspace, size_t workspace_bytes, int32_t* dev_status, void* stream) {
  return newton_step<mgs::DD>(J, ldj, F, x, m, n, tol, dev_state, workspace, workspace_bytes, dev_status, stream);
}
int newton_step_qd(double* J, int ldj, double* F, double* x, int m, int n, double tol, mgs_newton_state* dev_state,
                   void* workspace, size_t workspace_bytes, int32_t* dev_status, void* stream) {
  return newton_step<mgs::QD>(J, ldj, F, x, m, n, tol, dev_state, workspace, workspace_bytes, dev_status, stream);
}

}  // extern "C"
