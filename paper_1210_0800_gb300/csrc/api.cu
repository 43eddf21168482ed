// C ABI of the MGS least-squares library: argument checks, the Br x Bc decomposition,
// the workspace layout and the launch.  See include/mgs_ddqd.h for the contract.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/mgs_ddqd.h"
#include "launch.cuh"

namespace mgs {
int launch_cluster_d(const Params& pr, int grid, int cl, int T, size_t smem, cudaStream_t stream);
int launch_cluster_dd(const Params& pr, int grid, int cl, int T, size_t smem, cudaStream_t stream);
int launch_cluster_qd(const Params& pr, int grid, int cl, int T, size_t smem, cudaStream_t stream);
int cluster_capacity_d(int cl, int T, size_t smem);
int cluster_capacity_dd(int cl, int T, size_t smem);
int cluster_capacity_qd(int cl, int T, size_t smem);
int launch_cluster(int L, const Params& pr, int grid, int cl, int T, size_t smem, cudaStream_t stream) {
  return L == 1   ? launch_cluster_d(pr, grid, cl, T, smem, stream)
         : L == 2 ? launch_cluster_dd(pr, grid, cl, T, smem, stream)
                  : launch_cluster_qd(pr, grid, cl, T, smem, stream);
}
int cluster_capacity(int L, int cl, int T, size_t smem) {
  return L == 1 ? cluster_capacity_d(cl, T, smem) : L == 2 ? cluster_capacity_dd(cl, T, smem) : cluster_capacity_qd(cl, T, smem);
}
int blocks_per_sm_d(int kind, int T, size_t smem);
int blocks_per_sm_dd(int kind, int T, size_t smem);
int blocks_per_sm_qd(int kind, int T, size_t smem);
int grid_capacity(int L, int kind, int T, size_t smem) {
  return L == 1 ? blocks_per_sm_d(kind, T, smem) : L == 2 ? blocks_per_sm_dd(kind, T, smem) : blocks_per_sm_qd(kind, T, smem);
}
}  // namespace mgs

namespace {

thread_local int g_last_cuda = 0;

constexpr int kMaxBr = 32;             // partial reduction uses one warp-shuffle group
constexpr size_t kMaxSmem = 227 * 1024;  // dynamic shared memory per CTA on sm_103a
constexpr long long kTimeoutNs = 4000000000LL;  // 4 s: far above any legitimate wait

struct Plan {
  int L, m, n, nc, aug;
  int Br, Bc, h, w;
  int kind;  // 0 grid barrier per step, 1 hardware clusters, 2 software groups
  int T;     // threads per CTA (128 or 256)
  size_t smem;
  size_t off_sync, off_gsync, off_flags, off_P, off_V, off_Y, off_R, off_G, off_T, total, zero_bytes;
};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Dynamic shared memory that keeps more than `cps` CTAs off an SM (cps = 1: each CTA of the
// solve has the SM's FP64 unit to itself; cps = 2: two CTAs share it and hide each other's
// barrier and reduction latency).
size_t cta_per_sm_smem(int cps) {
  int dev = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess) return 0;
  return (size_t)per_sm / (size_t)(cps + 1);
}

int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return sms;
}

// Rows per CTA about 64; as many column groups as SMs allow; every row block non-empty.
bool compute_plan(int L, int m, int n, int aug, int want, int h0, int T0, int cps, Plan& pl) {
  if ((L != 1 && L != 2 && L != 4) || n < 1 || m < n) return false;
  const int sms = device_sms();
  if (sms <= 0) return false;
  pl.L = L;
  pl.m = m;
  pl.n = n;
  pl.aug = aug ? 1 : 0;
  pl.nc = n + pl.aug;
  const int E = 2 * L;
  // MGS_KERNEL = grid | cluster | group overrides the default choice: the cluster
  // schedule on hardware clusters for complex double and double-double (where the
  // per-step latency is a large share of a step) when the clusters fill at least 90 % of
  // the SMs a plain grid would use; otherwise, and for quad double (where the FP64
  // throughput decides), the grid-barrier kernel
  int h = h0;
  const size_t pad = cta_per_sm_smem(cps);
  auto padded = [&](size_t v) { return (pad > v && pad <= kMaxSmem) ? pad : v; };
  for (;;) {
    const int Br = (m + h - 1) / h;
    if (Br > kMaxBr || Br > sms) return false;
    const int Bc_grid = cps * sms / Br < pl.nc ? cps * sms / Br : pl.nc;
    if (Bc_grid < 1) return false;
    int kind = want < 0 ? (L <= 2 ? 1 : 0) : want, Bc = Bc_grid;
    // 256 threads (two warps per sub-partition) where a CTA owns many columns: their
    // long per-step loops then hide each other's FP64 latency
    const int T = T0 ? T0 : ((pl.nc + Bc_grid - 1) / Bc_grid >= 16 ? 256 : 128);
    if (kind == 1) {
      // hardware clusters: as many column groups as clusters fit at once
      int cap = 0;
      if (Br <= 8) {
        for (int it = 0, Bt = Bc_grid; it < 3; ++it) {
          const int wt = (pl.nc + Bt - 1) / Bt;
          cap = mgs::cluster_capacity(L, Br, T, padded(mgs::cluster_smem_bytes(L, h, wt, T)));
          if (cap <= 0 || Bt <= cap) break;
          Bt = cap;
        }
      }
      // by default only where the clusters occupy nearly as many SMs as a plain grid
      if (cap > 0 && (want == 1 || 10 * cap >= 9 * Bc_grid)) {
        Bc = cap < Bc_grid ? cap : Bc_grid;
      } else {
        kind = 0;
      }
    }
    const int w = (pl.nc + Bc - 1) / Bc;
    size_t smem = kind == 0 ? mgs::smem_bytes(L, h, w, T) : mgs::cluster_smem_bytes(L, h, w, T);
    const size_t bs = mgs::backsub_smem_bytes(L);
    if (bs > smem) smem = bs;
    if (smem <= kMaxSmem) {
      if (kind != 1 && mgs::grid_capacity(L, kind, T, padded(smem)) * sms < Br * Bc) return false;
      pl.Br = Br;
      pl.Bc = Bc;
      pl.h = h;
      pl.w = w;
      pl.smem = padded(smem);
      pl.kind = kind;
      pl.T = T;
      break;
    }
    if (h <= 8) return false;
    h /= 2;
  }
  size_t off = 0;
  pl.off_sync = off;
  off = align256(off + 64);
  pl.off_gsync = off;  // per-group arrival counters, 128 bytes apart
  off = align256(off + sizeof(unsigned) * 32 * (size_t)pl.Bc);
  pl.off_flags = off;
  off = align256(off + sizeof(int) * (size_t)(pl.nc + 1) * pl.Br);  // pivot-ready flags
  pl.zero_bytes = off;
  const int ACC = (L == 1) ? mgs::D::ACC : (L == 2) ? mgs::DD::ACC : mgs::QD::ACC;
  pl.off_P = off;
  const size_t pdoubles = pl.kind == 0 ? 2 * (size_t)pl.Br * pl.nc * ACC
                          : pl.kind == 2 ? mgs::group_partials_doubles(L, pl.Br, pl.Bc, (pl.nc + pl.Bc - 1) / pl.Bc)
                                         : 0;
  off = align256(off + sizeof(double) * pdoubles);
  pl.off_V = off;  // published pivot rows: a ring of Bc + 2 slots (cluster schedule), two otherwise
  off = align256(off + sizeof(double) * (size_t)(pl.kind != 0 ? pl.Bc + 2 : 2) * pl.Br * pl.h * E);
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

// The plan for (device, sizes, kernel choice), computed once: it queries occupancy, which
// costs far more host time than a launch.
bool make_plan(int L, int m, int n, int aug, Plan& pl) {
  struct Entry {
    int dev, L, m, n, aug, want, h, T, cps;
    Plan pl;
  };
  static std::mutex mu;
  static std::vector<Entry> cache;
  // MGS_KERNEL = grid | cluster | group, MGS_ROWS = h: overrides, read at every call
  const char* kenv = std::getenv("MGS_KERNEL");
  const int want = !kenv                          ? -1
                   : std::strcmp(kenv, "grid") == 0    ? 0
                   : std::strcmp(kenv, "cluster") == 0 ? 1
                   : std::strcmp(kenv, "group") == 0   ? 2
                                                       : -1;
  const char* henv = std::getenv("MGS_ROWS");
  int h = henv ? std::atoi(henv) : 64;
  if (h < 8 || h > 1024) h = 64;
  const char* tenv = std::getenv("MGS_CTA_THREADS");  // 128 | 256 (default: by layout)
  const int T = tenv && std::atoi(tenv) == 256 ? 256 : tenv && std::atoi(tenv) == 128 ? 128 : 0;
  const char* cenv = std::getenv("MGS_CTAS_PER_SM");  // 1 | 2 (default 1)
  const int cps = cenv && std::atoi(cenv) == 2 ? 2 : 1;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  {
    std::lock_guard<std::mutex> g(mu);
    for (const Entry& e : cache)
      if (e.dev == dev && e.L == L && e.m == m && e.n == n && e.aug == aug && e.want == want && e.h == h &&
          e.T == T && e.cps == cps) {
        pl = e.pl;
        return true;
      }
  }
  if (!compute_plan(L, m, n, aug, want, h, T, cps, pl)) return false;
  std::lock_guard<std::mutex> g(mu);
  if (cache.size() >= 256) cache.clear();
  cache.push_back(Entry{dev, L, m, n, aug, want, h, T, cps, pl});
  return true;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int run(int L, double* A, int lda, double* b, double* x, double* R, int ldr, double* z, int m, int n, void* ws,
        size_t ws_bytes, int32_t* dev_status, void* stream, int aug, const int32_t* skip = nullptr) {
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
  pr.gsync = reinterpret_cast<unsigned*>(wb + pl.off_gsync);
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
  pr.skip = skip;
#if defined(MGS_TRACE) && MGS_TRACE
  pr.trace = reinterpret_cast<unsigned long long*>(wb + pl.off_T);
#else
  pr.trace = nullptr;
#endif
  const int grid = pl.Br * pl.Bc;
  int rc;
  if (pl.kind == 1)
    rc = mgs::launch_cluster(L, pr, grid, pl.Br, pl.T, pl.smem, st);
  else
    rc = (L == 1) ? mgs::launch_d(pr, grid, pl.T, pl.smem, st, pl.kind)
         : (L == 2) ? mgs::launch_dd(pr, grid, pl.T, pl.smem, st, pl.kind)
                    : mgs::launch_qd(pr, grid, pl.T, pl.smem, st, pl.kind);
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
// The least-squares solve of ls_solve_*, doing nothing when *skip != 0 at launch time.
int ls_solve_gated(int L, double* A, int lda, double* b, double* x, double* z, int m, int n, void* ws,
                   size_t ws_bytes, int32_t* dev_status, void* stream, const int32_t* skip) {
  return run(L, A, lda, b, x, nullptr, 0, z, m, n, ws, ws_bytes, dev_status, stream, 1, skip);
}
}  // namespace mgs

extern "C" {

int mgs_version(void) { return 200; }

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

int mgs_plan_query(int limbs, int m, int n, int with_rhs, int* out) {
  if (!out || (limbs != 1 && limbs != 2 && limbs != 4) || m < 1 || n < 1 || m < n) return MGS_EINVAL;
  Plan pl;
  if (!make_plan(limbs, m, n, with_rhs, pl)) return MGS_ENOSPACE;
  out[0] = pl.Br;
  out[1] = pl.Bc;
  out[2] = pl.h;
  out[3] = pl.kind;
  out[4] = pl.T;
  return MGS_OK;
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
