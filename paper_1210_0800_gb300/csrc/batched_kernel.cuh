// Batched least squares: many independent complex DD/QD systems of different sizes in
// one launch (the pleasingly parallel case the paper sets aside when it tracks a single
// path, Section 2).  Each system is solved by one CTA with the method of Section 3
// (MGS on [A b], Figure 1 and Eq. 1) and Section 6 (back substitution, Figure 3).
//
// Organisation: CTAs take systems from a device work queue (an atomic counter over an
// optional order array, e.g. largest first); no CTA ever waits for another.  A system's
// matrix stays in global memory (L1/L2); the pivot column, the reduction tree and the
// coefficients are in shared memory.  Per step: Gram partials of all trailing columns
// against the pivot (one lane per (column, part, row chunk)), a shared-memory tree,
// c_kj = G_kj / G_kk, the update a_j -= c_kj a_k.  Normalisation and the scaled back
// substitution follow the single-system kernel.
//
// Split systems (S = 2 or 4, for batches smaller than the GPU): the S CTAs of a
// thread-block cluster share one system, each keeping a contiguous slice of its rows; the
// Gram partials of the slices are summed through distributed shared memory in rank order,
// so every CTA derives the same coefficients; the normalisation is split by rows and the
// back substitution runs on rank 0.
#pragma once

#include <cooperative_groups.h>

#include <cstdint>

#include "ddqd.cuh"
#include "mgs_kernel.cuh"

namespace mgs {

struct BatchParams {
  double* A;  // pool; system i at A + a_off[i] * 2L, column-major with leading dimension m_i
  double* b;  // pool; system i at b + b_off[i] * 2L (m_i elements)
  double* x;  // pool; system i at x + x_off[i] * 2L (n_i elements)
  const long long* a_off;
  const long long* b_off;
  const long long* x_off;
  const int* m_arr;
  const int* n_arr;
  const int* order;  // optional: the queue hands out order[0], order[1], ... (nullptr: 0, 1, ...)
  double* R;         // optional output: packed upper triangle of R, system i at R + r_off[i] * 2L
  const long long* r_off;
  int batch, max_m, max_n;
  unsigned* counter;  // work-queue head (zeroed before the launch)
  double* ws;         // per-CTA scratch, per_cta doubles each
  long long per_cta;
  int* status;  // one word per system
  int cmax;     // most lanes per (column, part) of a Gram row; 0 = no cap
  double one, nzero;
};

// Shared memory of one batched CTA (S CTAs per system).
__host__ __device__ inline size_t batched_smem_bytes(int L, int T, int max_m, int max_n, int S = 1) {
  const size_t E = 2 * (size_t)L;
  return sizeof(double) * ((size_t)max_m * E          // pivot column
                           + (size_t)(max_n + 1) * E  // coefficients / Gram row
                           + (size_t)T * L            // reduction tree
                           + 2 * E                    //
                           + (S > 1 ? 2 * (size_t)(max_n + 1) * 2 * L : 0))  // slice partials, 2 buffers
         + 16 * sizeof(int);
}

// Per-CTA global scratch (doubles): packed upper R (coefficients, then scaled columns),
// y, G_kk, r_kk, 1/r_kk.
__host__ __device__ inline long long batched_scratch_doubles(int L, int max_n) {
  const long long E = 2 * (long long)L, nc = max_n + 1;
  const long long v = (long long)max_n * (max_n + 1) / 2 * E + nc * E + 3 * nc * L;
  return (v + 31) / 32 * 32;
}

template <class Ar, int T, int S>
__global__ void __launch_bounds__(T) mgs_batched_kernel(BatchParams bp) {
  namespace cg = cooperative_groups;
  constexpr int L = Ar::L, E = 2 * L;
  using elem = typename Ar::elem;
  using real = typename Ar::real;
  using pacc = typename Ar::pacc;
  constexpr int PACC = Ar::PACC;
  static_assert(S == 1 || S == 2 || S == 4, "CTAs per system");
  const Fp f{bp.one, bp.nzero};
  const int tid = threadIdx.x;
  const int rank = (int)(blockIdx.x % S);  // the cluster is S consecutive CTAs
  const bool lead = rank == 0;

  extern __shared__ __align__(16) double sm[];
  double* piv = sm;                               // max_m * E, slice row l at l * E
  double* gbuf = piv + (size_t)bp.max_m * E;       // (max_n + 1) * E
  pacc* red = reinterpret_cast<pacc*>(gbuf + (size_t)(bp.max_n + 1) * E);  // T
  double* pslice = reinterpret_cast<double*>(red) + (size_t)T * L + 2 * E;  // S > 1: 2 x (max_n + 1) x 2 x PACC
  int* sflag = reinterpret_cast<int*>(pslice + (S > 1 ? 2 * (size_t)(bp.max_n + 1) * 2 * PACC : 0));
  // cluster barrier (S > 1): orders shared- and global-memory accesses of the S CTAs
  auto csync = [&]() {
    if constexpr (S > 1)
      cg::this_cluster().sync();
    else
      __syncthreads();
  };

  double* scr = bp.ws + (size_t)(blockIdx.x / S) * bp.per_cta;  // shared by the cluster
  double* Rp = scr;  // packed upper triangle: (k, j), k <= j, at (j (j + 1) / 2 + k) * E
  double* Yv = Rp + (size_t)bp.max_n * (bp.max_n + 1) / 2 * E;
  double* Gd = Yv + (size_t)(bp.max_n + 1) * E;
  double* Rd = Gd + (size_t)(bp.max_n + 1) * L;
  double* Ri = Rd + (size_t)(bp.max_n + 1) * L;

  auto ld_real = [&](const double* src) {
    real r;
    double* d = reinterpret_cast<double*>(&r);
#pragma unroll
    for (int q = 0; q < L; ++q) d[q] = src[q];
    return r;
  };
  auto st_real = [&](double* dst, const real& r) {
    const double* d = reinterpret_cast<const double*>(&r);
#pragma unroll
    for (int q = 0; q < L; ++q) dst[q] = d[q];
  };
  auto ld_part = [&](const double* p, int part) {
    elem e;
#pragma unroll
    for (int q = 0; q < E; ++q) e.v[q] = 0.0;
#pragma unroll
    for (int q = 0; q < L; ++q) e.v[part * L + q] = p[part * L + q];
    return e;
  };
  auto st_part = [&](double* p, const elem& e, int part) {
#pragma unroll
    for (int q = 0; q < L; ++q) p[part * L + q] = e.v[part * L + q];
  };
  auto packed = [](int k, int j) { return (size_t)j * (j + 1) / 2 + k; };

  for (;;) {
    csync();  // the cluster is done with the previous system
    if (tid == 0) {
      if (lead) sflag[0] = (int)atomicAdd(bp.counter, 1u);
      sflag[1] = ST_OK;
    }
    csync();
    int qi;
    if constexpr (S > 1) {
      qi = *cg::this_cluster().map_shared_rank(sflag, 0);
      csync();  // no CTA leaves while a peer still reads rank 0's shared memory
    } else {
      qi = sflag[0];
    }
    if (qi >= bp.batch) break;
    const int sys = bp.order ? bp.order[qi] : qi;
    const int m = bp.m_arr[sys], n = bp.n_arr[sys];
    if (n < 1 || m < n || m > bp.max_m || n > bp.max_n) {
      if (tid == 0) bp.status[sys] = ST_EINVAL;
      continue;
    }
    const int nc = n + 1;
    double* A = bp.A + (size_t)bp.a_off[sys] * E;
    double* bv = bp.b + (size_t)bp.b_off[sys] * E;
    double* xv = bp.x + (size_t)bp.x_off[sys] * E;
    auto col = [&](int j) -> double* { return (j < n) ? A + (size_t)j * m * E : bv; };
    // this CTA's slice of the rows
    const int mr = (m + S - 1) / S;
    const int r0 = min(m, rank * mr), ml = min(m, r0 + mr) - r0;
    // non-finite input check (own slice)
    {
      bool bad = false;
      for (int i = tid; i < ml * nc * E; i += T) {
        const int j = i / (ml * E), r = i % (ml * E);
        bad |= !finite64(col(j)[(size_t)r0 * E + r]);
      }
      if (bad) sflag[1] = ST_ENONFINITE;
    }
    __syncthreads();

    for (int k = 0; k < nc; ++k) {
      // pivot column rows of the slice
      for (int i = tid; i < ml * E; i += T) piv[i] = col(k)[(size_t)r0 * E + i];
      __syncthreads();
      // Gram row G_kj, j >= k: (column, part, row chunk) items; tree over chunks
      const int cols = nc - k, pairs = 2 * cols;
      double* pout = pslice + (size_t)(k & 1) * (bp.max_n + 1) * 2 * PACC;
      int C = T / pairs;
      if (bp.cmax > 0) C = min(C, bp.cmax);
      C = max(1, min(C, max(ml, 1)));
      const int per_round = T / C;
      for (int base = 0; base < pairs; base += per_round) {
        const int job = tid / C, ch = tid % C, pi = base + job;
        const bool act = job < per_round && pi < pairs;
        const int j = k + (pi >> 1), part = pi & 1;
        pacc a;
        Ar::pzero(a);
        if (act && !(j == k && part == 1)) {
          const double* cj = col(j) + (size_t)r0 * E;
          for (int l = ch; l < ml; l += C) {
            elem pe, ce;
#pragma unroll
            for (int q = 0; q < E; ++q) {
              pe.v[q] = piv[(size_t)l * E + q];
              ce.v[q] = cj[(size_t)l * E + q];
            }
            Ar::mac_part(f, a, pe, ce, part);
          }
        }
        red[tid] = a;
        __syncthreads();
        for (int st = 1; st < C; st <<= 1) {
          if (act && (ch % (2 * st)) == 0 && ch + st < C) {
            pacc x = red[tid];
            Ar::pcombine(f, x, red[tid + st]);
            red[tid] = x;
          }
          __syncthreads();
        }
        if (act && ch == 0) {
          if constexpr (S > 1) {
            const double* src = reinterpret_cast<const double*>(&red[tid]);
#pragma unroll
            for (int q = 0; q < PACC; ++q) pout[(size_t)pi * PACC + q] = src[q];
          } else {
            double* dst = gbuf + (size_t)(j - k) * E + part * L;
            if (j == k && part == 1) {
#pragma unroll
              for (int q = 0; q < L; ++q) dst[q] = 0.0;
            } else {
              Ar::pfinal(f, red[tid], dst);
            }
          }
        }
        __syncthreads();
      }
      if constexpr (S > 1) {
        // sum the S slices' partials in rank order (the same order in every CTA)
        cg::cluster_group cl = cg::this_cluster();
        cl.sync();
        for (int t = tid; t < pairs; t += T) {
          const int j = k + (t >> 1), part = t & 1;
          double* dst = gbuf + (size_t)(j - k) * E + part * L;
          if (j == k && part == 1) {
#pragma unroll
            for (int q = 0; q < L; ++q) dst[q] = 0.0;
            continue;
          }
          pacc a;
          Ar::pzero(a);
          for (int pr = 0; pr < S; ++pr) {
            const double* src = cl.map_shared_rank(pout, pr) + (size_t)t * PACC;
            pacc o;
            double* od = reinterpret_cast<double*>(&o);
#pragma unroll
            for (int q = 0; q < PACC; ++q) od[q] = src[q];
            Ar::pcombine(f, a, o);
          }
          Ar::pfinal(f, a, dst);
        }
        __syncthreads();
      }
      const real G = ld_real(gbuf);
      const bool okpiv = Ar::positive(G);
      if (lead && tid == 0) st_real(Gd + (size_t)k * L, G);
      if (k == nc - 1) break;  // the right-hand side: keep G (z^2); its column is the residual
      if (!okpiv && tid == 0) sflag[1] = (sflag[1] == ST_OK) ? ST_ERANK : sflag[1];
      // coefficients c_kj = G_kj / G_kk (j > k), stored as row k of R (or y_k)
      const double invG = Ar::inv_lead(G);
      for (int t = tid; t < 2 * (cols - 1); t += T) {
        const int j = k + 1 + (t >> 1), part = t & 1;
        double* g = gbuf + (size_t)(j - k) * E;
        const elem ge = ld_part(g, part);
        elem cc = ge;
        if (okpiv) {
          Ar::div_real_part(f, cc, ge, G, invG, part);
        } else {
#pragma unroll
          for (int q = 0; q < E; ++q) cc.v[q] = 0.0;
        }
        st_part(g, cc, part);
        if (lead) st_part((j < n) ? Rp + packed(k, j) * E : Yv + (size_t)k * E, cc, part);
      }
      __syncthreads();
      // update a_j -= c_kj a_k, j > k (one lane per (column, slice row, part))
      const int tot = (cols - 1) * ml * 2;
      for (int idx = tid; idx < tot; idx += T) {
        const int part = idx & 1, rest = idx >> 1;
        const int j = k + 1 + rest / ml, l = rest % ml;
        double* p = col(j) + (size_t)(r0 + l) * E;
        elem y = ld_part(p, part), cc, pe;
#pragma unroll
        for (int q = 0; q < E; ++q) {
          cc.v[q] = gbuf[(size_t)(j - k) * E + q];
          pe.v[q] = piv[(size_t)l * E + q];
        }
        Ar::update_part(f, y, cc, pe, part);
        st_part(p, y, part);
      }
      __syncthreads();
    }
    __syncthreads();
    // r_kk, 1/r_kk (rank 0, into the cluster's scratch)
    if (lead)
      for (int k = tid; k < nc; k += T) {
        const real r = Ar::sqrt(f, ld_real(Gd + (size_t)k * L));
        st_real(Rd + (size_t)k * L, r);
        if (Ar::positive(r)) st_real(Ri + (size_t)k * L, Ar::inv_real(f, r));
      }
    __threadfence();
    csync();
    // q_j = a_j / r_jj over the slice; the last column (b) is the residual and stays
    for (int idx = tid; idx < n * ml * 2; idx += T) {
      const int part = idx & 1, rest = idx >> 1;
      const int j = rest / ml, l = rest % ml;
      const real r = ld_real(Rd + (size_t)j * L);
      if (!Ar::positive(r)) continue;
      double* p = col(j) + (size_t)(r0 + l) * E;
      const elem a = ld_part(p, part);
      elem q = a;
      Ar::div_real_part(f, q, a, r, Ar::inv_lead(r), part);
      st_part(p, q, part);
    }
    // the rest is rank 0's: R, back substitution, x, status
    if (!lead) continue;
    // optional R output (packed upper triangle): r_kj = c_kj r_kk, real diagonal r_jj
    if (bp.R) {
      double* Ro = bp.R + (size_t)bp.r_off[sys] * E;
      for (int idx = tid; idx < n * (n + 1); idx += T) {
        const int part = idx & 1, pi = idx >> 1;
        int j = (int)((sqrt(1.0 + 8.0 * (double)pi) - 1.0) * 0.5);  // pi = j (j + 1) / 2 + k
        while (j * (j + 1) / 2 > pi) --j;
        while ((j + 1) * (j + 2) / 2 <= pi) ++j;
        const int k = pi - j * (j + 1) / 2;
        elem out;
        if (k == j) {
          out = Ar::from_real(ld_real(Rd + (size_t)j * L));
        } else {
          const elem c = ld_part(Rp + packed(k, j) * E, part);
          out = c;
          Ar::mul_real_part(f, out, c, ld_real(Rd + (size_t)k * L), part);
        }
        st_part(Ro + packed(k, j) * E, out, part);
      }
      __syncthreads();
    }
    // back substitution on the column-scaled system: t_jk = r_jk / r_kk with
    // r_jk = c_jk r_jj (so t_jk = c_jk r_jj / r_kk), y_k = c_kn r_kk
    for (int idx = tid; idx < n * (n - 1); idx += T) {
      const int part = idx & 1;
      const int pi = idx >> 1;
      int k = (int)((1.0 + sqrt(1.0 + 8.0 * (double)pi)) * 0.5);
      while (k * (k - 1) / 2 > pi) --k;
      while ((k + 1) * k / 2 <= pi) ++k;
      const int j = pi - k * (k - 1) / 2;  // j < k
      double* p = Rp + packed(j, k) * E;
      const elem c = ld_part(p, part);
      elem t = c;
      Ar::mul_real_part(f, t, c, ld_real(Rd + (size_t)j * L), part);
      const elem t2 = t;
      Ar::mul_real_part(f, t, t2, ld_real(Ri + (size_t)k * L), part);
      st_part(p, t, part);
    }
    for (int idx = tid; idx < 2 * n; idx += T) {
      const int k = idx >> 1, part = idx & 1;
      double* p = Yv + (size_t)k * E;
      const elem c = ld_part(p, part);
      elem y = c;
      Ar::mul_real_part(f, y, c, ld_real(Rd + (size_t)k * L), part);
      st_part(p, y, part);
    }
    __syncthreads();
    for (int k = n - 1; k >= 0; --k) {
      elem xk;
#pragma unroll
      for (int q = 0; q < E; ++q) xk.v[q] = Yv[(size_t)k * E + q];  // x~_k = y_k
      for (int t = tid; t < 2 * k; t += T) {
        const int j = t >> 1, part = t & 1;
        double* p = Yv + (size_t)j * E;
        elem y = ld_part(p, part), tt;
#pragma unroll
        for (int q = 0; q < E; ++q) tt.v[q] = Rp[packed(j, k) * E + q];
        Ar::update_part(f, y, tt, xk, part);
        st_part(p, y, part);
      }
      __syncthreads();
    }
    // x_k = x~_k / r_kk
    for (int idx = tid; idx < 2 * n; idx += T) {
      const int k = idx >> 1, part = idx & 1;
      const elem xt = ld_part(Yv + (size_t)k * E, part);
      const real r = ld_real(Rd + (size_t)k * L);
      elem xo = xt;
      Ar::div_real_part(f, xo, xt, r, Ar::inv_lead(r), part);
      st_part(xv + (size_t)k * E, xo, part);
    }
    __syncthreads();
    if (tid == 0) {
      // the input check comes first: a non-finite entry in any slice wins over the
      // rank deficiency it causes (the other flags are the same in every slice)
      int stv = sflag[1];
      if constexpr (S > 1)
        for (int pr = 1; pr < S; ++pr)
          if (*cg::this_cluster().map_shared_rank(sflag + 1, pr) == ST_ENONFINITE) stv = ST_ENONFINITE;
      bp.status[sys] = stv;
    }
  }
}

}  // namespace mgs

namespace mgs {

// Adjoint of batched least squares (see include/mgs_ddqd.h): per system, from the
// forward's Q, packed R, x and residual r and the incoming gradient G of x,
//   u = R^{-H} G, w = R^{-1} u, grad_b = Q u, grad_A = r w^H - grad_b x^H.
struct AdjParams {
  const double* Q;   // pool, as A of the forward
  const double* R;   // packed upper R pool
  const double* x;   // pool
  const double* r;   // residual pool (b of the forward after the solve)
  const double* G;   // gradient of x, pool like x
  double* gA;        // output, pool like A
  double* gb;        // output, pool like b
  const long long* a_off;
  const long long* r_off;
  const long long* b_off;
  const long long* x_off;
  const int* m_arr;
  const int* n_arr;
  const int* order;
  int batch, max_m, max_n;
  unsigned* counter;
  int* status;
  double one, nzero;
};

__host__ __device__ inline size_t adjoint_smem_bytes(int L, int max_n) {
  return sizeof(double) * (3 * (size_t)max_n * 2 * L + 2 * 2 * L) + 16 * sizeof(int);
}

template <class Ar, int T>
__global__ void __launch_bounds__(T) mgs_adjoint_kernel(AdjParams ap) {
  constexpr int L = Ar::L, E = 2 * L;
  using elem = typename Ar::elem;
  using real = typename Ar::real;
  using pacc = typename Ar::pacc;
  const Fp f{ap.one, ap.nzero};
  const int tid = threadIdx.x;
  extern __shared__ __align__(16) double sm[];
  double* gv = sm;                           // max_n * E: G, reduced in place
  double* uv = gv + (size_t)ap.max_n * E;    // max_n * E: u = R^{-H} G (kept)
  double* wv = uv + (size_t)ap.max_n * E;    // max_n * E: u reduced in place, then w
  int* sflag = reinterpret_cast<int*>(wv + (size_t)ap.max_n * E + 2 * E);

  auto ld_part = [&](const double* p, int part) {
    elem e;
#pragma unroll
    for (int q = 0; q < E; ++q) e.v[q] = 0.0;
#pragma unroll
    for (int q = 0; q < L; ++q) e.v[part * L + q] = p[part * L + q];
    return e;
  };
  auto st_part = [&](double* p, const elem& e, int part) {
#pragma unroll
    for (int q = 0; q < L; ++q) p[part * L + q] = e.v[part * L + q];
  };
  auto ld_elem = [&](const double* p) {
    elem e;
#pragma unroll
    for (int q = 0; q < E; ++q) e.v[q] = p[q];
    return e;
  };
  auto packed = [](int k, int j) { return (size_t)j * (j + 1) / 2 + k; };

  for (;;) {
    __syncthreads();
    if (tid == 0) {
      sflag[0] = (int)atomicAdd(ap.counter, 1u);
      sflag[1] = ST_OK;
    }
    __syncthreads();
    const int qi = sflag[0];
    if (qi >= ap.batch) break;
    const int sys = ap.order ? ap.order[qi] : qi;
    const int m = ap.m_arr[sys], n = ap.n_arr[sys];
    if (n < 1 || m < n || m > ap.max_m || n > ap.max_n) {
      if (tid == 0) ap.status[sys] = ST_EINVAL;
      continue;
    }
    const double* Q = ap.Q + (size_t)ap.a_off[sys] * E;
    const double* R = ap.R + (size_t)ap.r_off[sys] * E;
    const double* xv = ap.x + (size_t)ap.x_off[sys] * E;
    const double* rv = ap.r + (size_t)ap.b_off[sys] * E;
    const double* Gv = ap.G + (size_t)ap.x_off[sys] * E;
    double* gA = ap.gA + (size_t)ap.a_off[sys] * E;
    double* gb = ap.gb + (size_t)ap.b_off[sys] * E;
    auto rdiag = [&](int k) {
      real r;
      double* d = reinterpret_cast<double*>(&r);
#pragma unroll
      for (int q = 0; q < L; ++q) d[q] = R[packed(k, k) * E + q];
      return r;
    };
    for (int i = tid; i < n * E; i += T) gv[i] = Gv[i];
    __syncthreads();
    // u = R^{-H} G: for k = 0..n-1, u_k = g_k / r_kk, then g_j -= conj(r_kj) u_k (j > k)
    for (int k = 0; k < n; ++k) {
      const real rk = rdiag(k);
      if (!Ar::positive(rk)) {
        if (tid == 0) sflag[1] = ST_ERANK;
      }
      if (tid < 2) {
        const elem g = ld_part(gv + (size_t)k * E, tid);
        elem u = g;
        Ar::div_real_part(f, u, g, rk, Ar::inv_lead(rk), tid);
        st_part(uv + (size_t)k * E, u, tid);
        st_part(wv + (size_t)k * E, u, tid);
      }
      __syncthreads();
      const elem uk = ld_elem(uv + (size_t)k * E);
      for (int t = tid; t < 2 * (n - 1 - k); t += T) {
        const int j = k + 1 + (t >> 1), part = t & 1;
        elem c = ld_elem(R + packed(k, j) * E);
#pragma unroll
        for (int q = 0; q < L; ++q) c.v[L + q] = flip_if(c.v[L + q], true);  // conj(r_kj)
        elem g = ld_part(gv + (size_t)j * E, part);
        Ar::update_part(f, g, c, uk, part);
        st_part(gv + (size_t)j * E, g, part);
      }
      __syncthreads();
    }
    // w = R^{-1} u: for k = n-1..0, w_k = u_k / r_kk, then u_j -= r_jk w_k (j < k);
    // wv holds u and is reduced in place, w_k replacing u_k
    for (int k = n - 1; k >= 0; --k) {
      const real rk = rdiag(k);
      if (tid < 2) {
        const elem y = ld_part(wv + (size_t)k * E, tid);
        elem w = y;
        Ar::div_real_part(f, w, y, rk, Ar::inv_lead(rk), tid);
        st_part(wv + (size_t)k * E, w, tid);
      }
      __syncthreads();
      const elem wk = ld_elem(wv + (size_t)k * E);
      for (int t = tid; t < 2 * k; t += T) {
        const int j = t >> 1, part = t & 1;
        elem y = ld_part(wv + (size_t)j * E, part);
        Ar::update_part(f, y, ld_elem(R + packed(j, k) * E), wk, part);
        st_part(wv + (size_t)j * E, y, part);
      }
      __syncthreads();
    }
    // grad_b = Q u: one lane per (row, part)
    for (int t = tid; t < 2 * m; t += T) {
      const int i = t >> 1, part = t & 1;
      pacc a;
      Ar::pzero(a);
      for (int k = 0; k < n; ++k) Ar::mul_acc_part(f, a, ld_elem(Q + ((size_t)k * m + i) * E), ld_elem(uv + (size_t)k * E), part);
      Ar::pfinal(f, a, gb + (size_t)i * E + part * L);
    }
    __syncthreads();
    // grad_A = r w^H - grad_b x^H, element (i, j): r_i conj(w_j) - g_i conj(x_j)
    for (int t = tid; t < 2 * m * n; t += T) {
      const int part = t & 1, rest = t >> 1;
      const int j = rest / m, i = rest % m;
      elem xn = ld_elem(xv + (size_t)j * E);
#pragma unroll
      for (int q = 0; q < E; ++q) xn.v[q] = flip_if(xn.v[q], true);
      pacc a;
      Ar::pzero(a);
      Ar::mac_part(f, a, ld_elem(wv + (size_t)j * E), ld_elem(rv + (size_t)i * E), part);
      Ar::mac_part(f, a, xn, ld_elem(gb + (size_t)i * E), part);
      Ar::pfinal(f, a, gA + ((size_t)j * m + i) * E + part * L);
    }
    __syncthreads();
    if (tid == 0) ap.status[sys] = sflag[1];
  }
}

}  // namespace mgs
