// Persistent modified Gram-Schmidt least-squares kernel (complex DD / QD) for sm_103a.
//
// Method (Verschelde & Yoffe):
//   Section 3, Figure 1 -- MGS: r_kk = ||a_k||, q_k = a_k / r_kk, r_kj = q_k^H a_j,
//                           a_j -= r_kj q_k for j > k;
//   Section 3, Eq. (1)  -- MGS on the augmented [A b]: the last column ends as the
//                           residual b - A x, its norm is z, and r_{k,n+1} = y_k = (Q^H b)_k;
//   Section 6, Figure 3 -- back substitution R x = y, column by column.
//
// GPU organisation (not the paper's per-step launches): one cooperative launch of
// Br x Bc CTAs that stays resident for the whole solve.
//   * CTA (p, c) owns rows [p h, p h + h) of the augmented columns j = c, c + Bc, ...
//     (column-cyclic, so every CTA keeps work as the trailing matrix shrinks) and keeps
//     that tile in shared memory from the first step to the last.
//   * Step k needs the Gram row G_kj = a_k^H a_j (j >= k) of the current columns; every
//     CTA writes its row-block partials, one grid barrier, every CTA reduces the Br
//     partials of the columns it owns (and of the pivot norm G_kk, identically everywhere).
//     The update is a_j -= (G_kj / G_kk) a_k, i.e. r_kj q_k with r_kj = G_kj / r_kk and
//     q_k = a_k / r_kk, so the pivot's square root and division stay off the update path.
//   * Look-ahead: the owners of column k+1 update it first and publish its rows through a
//     per-(step, row-block) flag; the other CTAs update their own columns meanwhile, then
//     read the new pivot and form the partials of step k+1.  One grid barrier per step.
//   * Deferred normalisation: during the sweep only G_kk and c_kj = G_kj / G_kk are needed;
//     the square roots r_kk, the columns q_k = a_k / r_kk and r_kj = c_kj r_kk are formed
//     once at the end, in parallel over all columns, from the unnormalised columns each
//     CTA still holds.  On the critical path of a step there is then one division.
//   * An FP64 instruction costs 64 cycles of the sub-partition's FP64 unit, so the latency
//     chains of a step (coefficients, the look-ahead column) split the real and imaginary
//     parts over two lanes.
//   * Every spin-wait gives up after a time limit, records a timeout status and lets the
//     remaining barriers fall through, so a missing CTA can never hang the GPU.
#pragma once

#include <cstdint>

#include "ddqd.cuh"

namespace mgs {

enum : int { ST_OK = 0, ST_EINVAL = 1, ST_ERANK = 2, ST_ENONFINITE = 3, ST_ETIMEOUT = 4 };

// Threads per CTA of the single-system kernels: 128 (one warp per SM sub-partition) or 256
// (two), a template parameter chosen per layout by the plan.

struct Params {
  double* A;  // m x n, column-major by element, leading dimension lda (elements); Q on exit
  long long lda;
  double* b;  // m elements (augmented column) or nullptr for a plain QR
  double* R;  // n x n, leading dimension ldr (elements)
  long long ldr;
  double* Rt;  // n x n (leading dimension n) scaled columns r_jk / r_kk for back substitution;
               // the same memory as R when the caller does not want R
  double* x;  // n elements (solution) or nullptr
  double* z;  // L doubles (residual norm) or nullptr
  int m, n, nc, aug;
  int Br, Bc, h;
  unsigned* sync;  // [0] barrier arrivals, [1] abort flag
  unsigned* gsync;  // per-column-group arrival counters, 32 apart (group kernel)
  int* flags;      // nc * Br pivot-ready flags
  double* P;       // partial Gram rows: 2 * Br * nc * ACC (group kernel: its partial buffers)
  double* V;       // published pivot rows: 2 (grid kernel) or Bc + 2 (cluster schedule) slots of Br * h * 2L
  double* Y;       // y = Q^H b (and the back-substitution right-hand side): nc * 2L
  double* Gd;      // pivot norms G_kk = ||a_k||^2: nc * L
  double* Rd;      // r_kk: nc * L
  double* Ri;      // 1 / r_kk: nc * L
  int* status;
  double one, nzero;
  long long timeout_ns;
  unsigned long long* trace;  // phase timestamps, (nc + 1) x grid x 8 (trace builds only)
  const int* skip;            // when non-null and nonzero at launch the kernel does nothing
};

// Phase timestamps for performance analysis (compiled in with -DMGS_TRACE=1 only).
#if defined(MGS_TRACE) && MGS_TRACE
#define MGS_TR(step, ph)                                                                    \
  do {                                                                                     \
    if (threadIdx.x == 0 && pr.trace)                                                      \
      pr.trace[((size_t)(step) * gridDim.x + blockIdx.x) * 8 + (ph)] = globaltimer();       \
  } while (0)
// the SM a CTA runs on (slot 7 of the step-0 record)
#define MGS_TR_SMID()                                                                       \
  do {                                                                                     \
    if (threadIdx.x == 0 && pr.trace) {                                                    \
      unsigned sid;                                                                        \
      asm volatile("mov.u32 %0, %%smid;" : "=r"(sid));                                     \
      pr.trace[(size_t)blockIdx.x * 8 + 7] = sid;                                          \
    }                                                                                      \
  } while (0)
#else
#define MGS_TR(step, ph) \
  do {                   \
  } while (0)
#define MGS_TR_SMID() \
  do {                \
  } while (0)
#endif

// ------------------------------------------------------------------ memory-model helpers
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_acquire_s32(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_s32(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void set_status(int* status, int code) { atomicCAS(status, ST_OK, code); }

// Grid-wide barrier on a monotone arrival counter.  Returns after all CTAs arrived, or
// after the abort flag is seen, or after the time limit (then it raises the abort flag).
// The last CTA to arrive learns it from its own atomic and does not poll; the others poll
// the counter alone and look at the abort flag and the clock every 64 polls, so the
// common path costs one memory round trip per poll.
__device__ __forceinline__ void grid_barrier(const Params& pr, unsigned& epoch) {
  __syncthreads();
  if (threadIdx.x == 0) {
    ++epoch;
    const unsigned target = epoch * gridDim.x;
    __threadfence();
    const unsigned arrived = atomicAdd(&pr.sync[0], 1u) + 1u;
    if (arrived < target) {
      const unsigned long long t0 = globaltimer();
      unsigned spins = 0;
      while (ld_acquire_u32(&pr.sync[0]) < target) {
        if ((++spins & 63u) == 0) {
          if (ld_acquire_u32(&pr.sync[1])) break;
          if ((long long)(globaltimer() - t0) > pr.timeout_ns) {
            set_status(pr.status, ST_ETIMEOUT);
            atomicExch(&pr.sync[1], 1u);
            break;
          }
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// Wait until flags[i] != 0 (bounded).  Called by one thread.  The flag is polled alone;
// the abort flag and the clock are looked at every 64 polls.
__device__ __forceinline__ void wait_flag(const Params& pr, const int* flag) {
  const unsigned long long t0 = globaltimer();
  unsigned spins = 0;
  while (ld_acquire_s32(flag) == 0) {
    if ((++spins & 63u) == 0) {
      if (ld_acquire_u32(&pr.sync[1])) return;
      if ((long long)(globaltimer() - t0) > pr.timeout_ns) {
        set_status(pr.status, ST_ETIMEOUT);
        atomicExch(&pr.sync[1], 1u);
        return;
      }
    }
  }
}

// ------------------------------------------------------------------ tile access
// Shared-memory planes: element (slot s, row l) limb q at base[(s * E + q) * h + l].
template <class Ar>
__device__ __forceinline__ typename Ar::elem sm_load(const double* base, int h, int l) {
  typename Ar::elem e;
#pragma unroll
  for (int q = 0; q < 2 * Ar::L; ++q) e.v[q] = base[q * h + l];
  return e;
}
template <class Ar>
__device__ __forceinline__ void sm_store(double* base, int h, int l, const typename Ar::elem& e) {
#pragma unroll
  for (int q = 0; q < 2 * Ar::L; ++q) base[q * h + l] = e.v[q];
}
// Only the limbs of one part (0 real, 1 imaginary); the other part reads as zero.  Lanes
// that own different parts of one element then never touch each other's limbs.
template <class Ar>
__device__ __forceinline__ typename Ar::elem sm_load_part(const double* base, int h, int l, int part) {
  typename Ar::elem e;
#pragma unroll
  for (int q = 0; q < 2 * Ar::L; ++q) e.v[q] = 0.0;
#pragma unroll
  for (int q = 0; q < Ar::L; ++q) e.v[part * Ar::L + q] = base[(part * Ar::L + q) * h + l];
  return e;
}
// Global element: 2L consecutive doubles, 16-byte aligned.
template <class Ar>
__device__ __forceinline__ typename Ar::elem g_load(const double* p) {
  typename Ar::elem e;
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int i = 0; i < Ar::L; ++i) {
    const double2 v = q[i];
    e.v[2 * i] = v.x;
    e.v[2 * i + 1] = v.y;
  }
  return e;
}
template <class Ar>
__device__ __forceinline__ typename Ar::elem g_load_cg(const double* p) {
  typename Ar::elem e;
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int i = 0; i < Ar::L; ++i) {
    const double2 v = __ldcg(q + i);
    e.v[2 * i] = v.x;
    e.v[2 * i + 1] = v.y;
  }
  return e;
}
template <class Ar>
__device__ __forceinline__ void g_store(double* p, const typename Ar::elem& e) {
  double2* q = reinterpret_cast<double2*>(p);
#pragma unroll
  for (int i = 0; i < Ar::L; ++i) q[i] = make_double2(e.v[2 * i], e.v[2 * i + 1]);
}
template <class Ar>
__device__ __forceinline__ void acc_store(double* p, const typename Ar::acc& a) {
  static_assert(sizeof(typename Ar::acc) == Ar::ACC * sizeof(double), "acc layout");
  const double* s = reinterpret_cast<const double*>(&a);
#pragma unroll
  for (int i = 0; i < Ar::ACC; ++i) p[i] = s[i];
}
template <class Ar>
__device__ __forceinline__ typename Ar::acc acc_load_cg(const double* p) {
  typename Ar::acc a;
  double* s = reinterpret_cast<double*>(&a);
#pragma unroll
  for (int i = 0; i < Ar::ACC; ++i) s[i] = __ldcg(p + i);
  return a;
}
template <class Ar>
__device__ __forceinline__ typename Ar::acc acc_shfl_xor(const typename Ar::acc& a, int mask) {
  typename Ar::acc r;
  const double* s = reinterpret_cast<const double*>(&a);
  double* d = reinterpret_cast<double*>(&r);
#pragma unroll
  for (int i = 0; i < Ar::ACC; ++i) d[i] = __shfl_xor_sync(0xffffffffu, s[i], mask);
  return r;
}

__device__ __forceinline__ int pow2_floor(int v) { return v <= 1 ? 1 : 1 << (31 - __clz(v)); }
__device__ __forceinline__ int pow2_ceil(int v) { return v <= 1 ? 1 : 1 << (32 - __clz(v - 1)); }
__device__ __forceinline__ int ceil_log2(int v) { return v <= 1 ? 0 : 32 - __clz(v - 1); }

// Partials of one step: `pairs` (column, part) dot products over hr rows.  The strided
// mapping gives each pair C lanes (rows ch, ch + C, ...) and a tree of log2 C levels;
// the flat mapping gives every lane the same number of consecutive (pair, row) items.
// A warp pays for every FP64 instruction whatever its active lanes, so the mapping with
// fewer products plus combines on the busiest lane wins.  The flat one needs a lane's
// items to span at most two pairs, i.e. pairs <= T.
template <class Ar, int T>
__device__ __forceinline__ bool flat_partials_cheaper(int pairs, int hr, int C) {
  if (pairs > T || hr < 1) return false;
  const int per_round = T / C;
  const int rounds = (pairs + per_round - 1) / per_round;
  const int strided = rounds * (((hr + C - 1) / C) * Ar::kMacOps + ceil_log2(C) * Ar::kCombineOps);
  const int per = (pairs * hr + T - 1) / T;
  const int flat = per * Ar::kMacOps + (ceil_log2((hr + per - 1) / per) + 1) * Ar::kCombineOps;
  return flat < strided;
}

// a_j -= c_j p for the tile slots [sb, sb + nb) over the CTA's hr rows (c_j at
// coef + slot * 2L, the pivot rows in piv).  For D and DD with at least two elements per
// thread a lane takes a whole element: its two parts are independent dependency chains the
// FP64 pipe interleaves, and the element is loaded once (measured: +1-3 %; for QD the
// doubled register state costs more than it gains).  Otherwise one lane per element part
// keeps every lane busy.  Both mappings perform the same operations on every part.
template <class Ar, int T>
__device__ __forceinline__ void update_slots(const Fp& f, double* tile, const double* coef, const double* piv, int h,
                                             int hr, int sb, int nb) {
  constexpr int L = Ar::L, E = 2 * L;
  using elem = typename Ar::elem;
  const int tid = threadIdx.x;
  if (nb <= 0 || hr <= 0) return;
  const int elems = nb * hr;
  if (L <= 2 && elems >= 2 * T) {
    for (int idx = tid; idx < elems; idx += T) {
      const int s = sb + idx / hr, l = idx % hr;
      double* ts = tile + (size_t)s * E * h;
      elem cc;
#pragma unroll
      for (int q = 0; q < E; ++q) cc.v[q] = coef[(size_t)s * E + q];
      elem y = sm_load<Ar>(ts, h, l);
      Ar::update(f, y, cc, sm_load<Ar>(piv, h, l));
      sm_store<Ar>(ts, h, l, y);
    }
  } else {
    for (int idx = tid; idx < 2 * elems; idx += T) {
      const int part = idx & 1, rest = idx >> 1;
      const int s = sb + rest / hr, l = rest % hr;
      double* ts = tile + (size_t)s * E * h;
      elem cc;
#pragma unroll
      for (int q = 0; q < E; ++q) cc.v[q] = coef[(size_t)s * E + q];
      elem y = sm_load_part<Ar>(ts, h, l, part);
      Ar::update_part(f, y, cc, sm_load<Ar>(piv, h, l), part);
#pragma unroll
      for (int q = 0; q < L; ++q) ts[(part * L + q) * h + l] = y.v[part * L + q];
    }
  }
}

// Shared-memory footprint (bytes) of one CTA.
__host__ __device__ inline size_t smem_bytes(int L, int h, int w, int T) {
  const size_t E = 2 * (size_t)L;
  return sizeof(double) * ((size_t)(w + 2) * E * h  // tile + two pivot buffers
                           + (size_t)(w + 1) * E     // coefficients + pivot norm
                           + 4 * E                   // scalars
                           + (size_t)T * L)          // partial-sum reduction tree
         + 16 * sizeof(int);
}

// Back substitution block size (rows of R solved by one CTA between grid barriers).
constexpr int kBS = 32;
// Shared memory of the back substitution's diagonal block: right-hand side and t_jk.
__host__ __device__ inline size_t backsub_smem_bytes(int L) {
  return sizeof(double) * (size_t)(kBS + kBS * kBS) * 2 * L + 64;
}

// Normalisation (Q = a_k / r_kk from the CTA's resident tile, R = c r_kk), then the
// back substitution; shared by the single-system kernels.  The tile layout is the one
// both kernels keep in shared memory: slot s of column c + s Bc, limb planes of h rows.
template <class Ar, int T>
__device__ __forceinline__ void mgs_epilogue(const Params& pr, unsigned& epoch, double* sm, int p, int c) {
  constexpr int L = Ar::L, E = 2 * L;
  using elem = typename Ar::elem;
  using real = typename Ar::real;
  using pacc = typename Ar::pacc;
  constexpr int PACC = Ar::PACC;
  const Fp f{pr.one, pr.nzero};
  const int tid = threadIdx.x;
  const int Bc = pr.Bc, Br = pr.Br, nc = pr.nc, h = pr.h;
  const int r0 = p * h;
  const int hr = max(0, min(h, pr.m - r0));
  const int w = (nc - c + Bc - 1) / Bc;
  double* tile = sm;
  auto col_of = [&](int s) { return c + s * Bc; };
  auto ld_real = [&](const double* src) {
    real r;
    double* d = reinterpret_cast<double*>(&r);
#pragma unroll
    for (int q = 0; q < L; ++q) d[q] = __ldcg(src + q);
    return r;
  };
  auto st_real = [&](double* dst, const real& r) {
    const double* d = reinterpret_cast<const double*>(&r);
#pragma unroll
    for (int q = 0; q < L; ++q) dst[q] = d[q];
  };
  // ---------------------------------------------------------------- normalisation
  const int nthreads = gridDim.x * T;
  const int gtid = blockIdx.x * T + tid;
  // (E1) r_kk = sqrt(G_kk) and 1 / r_kk for every column, spread over all threads
  for (int k = gtid; k < nc; k += nthreads) {
    const real G = ld_real(pr.Gd + (size_t)k * L);
    const real r = Ar::sqrt(f, G);
    st_real(pr.Rd + (size_t)k * L, r);
    if (Ar::positive(r)) st_real(pr.Ri + (size_t)k * L, Ar::inv_real(f, r));
    if (pr.aug && k == nc - 1 && pr.z) st_real(pr.z, r);
  }
  grid_barrier(pr, epoch);
  MGS_TR(nc, 1);
  // (E2) q_j = a_j / r_jj for the own columns (the tile holds the unnormalised columns)
  {
    const int nq = pr.n;  // columns that are normalised
    const int wq = (nq - c + Bc - 1) / Bc;
    if (wq > 0 && hr > 0) {
      const int tot = wq * hr * 2;
      for (int idx = tid; idx < tot; idx += T) {
        const int part = idx & 1, rest = idx >> 1;
        const int s = rest / hr, l = rest % hr, j = col_of(s);
        const real r = ld_real(pr.Rd + (size_t)j * L);
        if (!Ar::positive(r)) continue;
        const elem a = sm_load<Ar>(tile + (size_t)s * E * h, h, l);
        elem q = a;
        Ar::div_real_part(f, q, a, r, Ar::inv_lead(r), part);
#pragma unroll
        for (int qq = 0; qq < L; ++qq) pr.A[((size_t)j * pr.lda + r0 + l) * E + part * L + qq] = q.v[part * L + qq];
      }
    }
  }
  // (E3) r_kj = c_kj r_kk for the own columns (rows k < j split over the row blocks),
  //      y_k = c_kn r_kk, and the real diagonal r_jj
  {
    for (int s = 0; s < w; ++s) {
      const int j = col_of(s);
      const int tot = j * 2;  // (k, part) pairs with k < j
      for (int idx = p * T + tid; idx < tot; idx += Br * T) {
        const int k = idx >> 1, part = idx & 1;
        double* dst = (j < pr.n) ? pr.R + ((size_t)j * pr.ldr + k) * E : pr.Y + (size_t)k * E;
        elem cc;
#pragma unroll
        for (int q = 0; q < E; ++q) cc.v[q] = 0.0;
#pragma unroll
        for (int q = 0; q < L; ++q) cc.v[part * L + q] = __ldcg(dst + part * L + q);
        elem r = cc;
        Ar::mul_real_part(f, r, cc, ld_real(pr.Rd + (size_t)k * L), part);
#pragma unroll
        for (int q = 0; q < L; ++q) dst[part * L + q] = r.v[part * L + q];
      }
      if (p == 0 && tid == 0 && j < pr.n) g_store<Ar>(pr.R + ((size_t)j * pr.ldr + j) * E,
                                                     Ar::from_real(ld_real(pr.Rd + (size_t)j * L)));
    }
  }

  // ---------------------------------------------------------------- back substitution
  if (!pr.aug || pr.x == nullptr) return;
  grid_barrier(pr, epoch);
  // Figure 3 on the column-scaled system: with D = diag(r_kk), R x = y is solved as
  // (R D^-1)(D x) = y.  The scaled columns t_jk = r_jk / r_kk are formed once, in parallel;
  // the sequential chain is then x~_k = y_k and y_j -= t_jk x~_k (one update per link
  // instead of a product and an update), and x_k = x~_k / r_kk (a true division) for all k
  // in parallel at the end.
  const int n = pr.n;
  {
    const long long tot = (long long)n * (n - 1);  // (j < k) pairs x 2 parts
    for (long long idx = gtid; idx < tot; idx += nthreads) {
      const int part = (int)(idx & 1);
      const long long pi = idx >> 1;
      int k = (int)((1.0 + sqrt(1.0 + 8.0 * (double)pi)) * 0.5);  // pi = k(k-1)/2 + j
      while ((long long)k * (k - 1) / 2 > pi) --k;
      while ((long long)(k + 1) * k / 2 <= pi) ++k;
      const int j = (int)(pi - (long long)k * (k - 1) / 2);
      elem r;
#pragma unroll
      for (int q = 0; q < E; ++q) r.v[q] = 0.0;
#pragma unroll
      for (int q = 0; q < L; ++q) r.v[part * L + q] = __ldcg(pr.R + ((size_t)k * pr.ldr + j) * E + part * L + q);
      elem t = r;
      Ar::mul_real_part(f, t, r, ld_real(pr.Ri + (size_t)k * L), part);
#pragma unroll
      for (int q = 0; q < L; ++q) pr.Rt[((size_t)k * n + j) * E + part * L + q] = t.v[part * L + q];
    }
  }
  grid_barrier(pr, epoch);
  if constexpr (L == 4) {
    // QD: within each diagonal block the unknowns go in pairs (k, k-1), k = e-1, e-3, ...
    // The lower row of a pair is replaced by itself minus t_{k-1,k} times the upper row,
    // which eliminates t_{k-1,k}: s_{k-1,m} = t_{k-1,m} - t_{k-1,k} t_{k,m} for m > k in
    // the block (written over t_{k-1,m}; every operand is an entry this pass leaves alone).
    // The chain then yields two unknowns per link (see below).
    const int nblk = (n + kBS - 1) / kBS;
    const long long tot = (long long)nblk * kBS * kBS * 2;
    for (long long idx = gtid; idx < tot; idx += nthreads) {
      const int part = (int)(idx & 1);
      const long long r = idx >> 1;
      const int mm = (int)(r % kBS), jj = (int)((r / kBS) % kBS), bk = (int)(r / ((long long)kBS * kBS));
      const int e = n - bk * kBS, sb = max(0, e - kBS), nbk = e - sb;
      if (jj >= nbk || mm >= nbk || mm < jj + 2 || ((nbk - jj) & 1)) continue;
      const int j = sb + jj, m = sb + mm;
      double* dst = pr.Rt + ((size_t)m * n + j) * E;
      elem t;
#pragma unroll
      for (int q = 0; q < E; ++q) t.v[q] = 0.0;
#pragma unroll
      for (int q = 0; q < L; ++q) t.v[part * L + q] = __ldcg(dst + part * L + q);
      Ar::update_part(f, t, g_load_cg<Ar>(pr.Rt + ((size_t)(j + 1) * n + j) * E),
                      g_load_cg<Ar>(pr.Rt + ((size_t)m * n + j + 1) * E), part);
#pragma unroll
      for (int q = 0; q < L; ++q) dst[part * L + q] = t.v[part * L + q];
    }
    grid_barrier(pr, epoch);
  }
  MGS_TR(nc, 2);
  // blocks of kBS rows: CTA 0 runs the chain of the diagonal block (its t_jk staged in
  // shared memory), then every CTA applies the block's x~ to the rows above it.
  for (int e = n; e > 0; e -= kBS) {
    const int s = max(0, e - kBS);
    const int nbk = e - s;
    if (blockIdx.x == 0) {
      double* ys = sm;                          // nbk * E, row k at (k - s) * E
      double* tb = sm + (size_t)kBS * E;        // t_jk (j < k in the block) at ((k - s) kBS + j - s) E
      for (int i = tid; i < nbk; i += T) {
        const elem v = g_load_cg<Ar>(pr.Y + (size_t)(s + i) * E);
#pragma unroll
        for (int q = 0; q < E; ++q) ys[(size_t)i * E + q] = v.v[q];
      }
      for (int i = tid; i < nbk * nbk; i += T) {
        const int kk = i / nbk, jj = i % nbk;
        if (jj >= kk) continue;
        const elem v = g_load_cg<Ar>(pr.Rt + ((size_t)(s + kk) * n + s + jj) * E);
#pragma unroll
        for (int q = 0; q < E; ++q) tb[((size_t)kk * kBS + jj) * E + q] = v.v[q];
      }
      __syncthreads();
      if constexpr (L == 4) {
        // QD, pairs (k, k-1): first w_{k-1} = y_{k-1} - t_{k-1,k} y_k for every pair (the
        // lower rows' coefficients are the eliminated s_{k-1,m}).  A link then takes
        // x~_k = y_k and x~_{k-1} = w_{k-1} together and subtracts both terms from every
        // row below: per row and part one lane per term (two QD products, the first lane
        // seeded with y_j), merged through a shuffle.  Half the links of the one-unknown
        // chain, each about 183 FP64 instructions instead of 2 x 113.
        static_assert(4 * (kBS - 2) <= T, "one pass of a pair link");
        const int np = nbk / 2;
        {
          const int t = tid;
          const bool act = t < 4 * np;
          const int pi = t >> 2, part = (t >> 1) & 1, half = t & 1;
          const int k = e - 1 - 2 * pi;
          double* yw = ys + (size_t)(act ? k - 1 - s : 0) * E;
          pacc a;
          Ar::pzero(a);
          if (act) {
            if (half == 0) Ar::pseed(a, yw + part * L);
            Ar::mul_sub_half(f, a, sm_load<Ar>(tb + ((size_t)(k - s) * kBS + (k - 1 - s)) * E, 1, 0),
                             sm_load<Ar>(ys + (size_t)(k - s) * E, 1, 0), part, half);
          }
          pacc o;
          const double* sa = reinterpret_cast<const double*>(&a);
          double* so = reinterpret_cast<double*>(&o);
#pragma unroll
          for (int q = 0; q < PACC; ++q) so[q] = __shfl_xor_sync(0xffffffffu, sa[q], 1);
          if (act && half == 0) {
            Ar::pcombine(f, a, o);
            Ar::pfinal(f, a, yw + part * L);
          }
          __syncthreads();
        }
        for (int k = e - 1; k - 1 >= s; k -= 2) {
          elem xk, xk1;
#pragma unroll
          for (int q = 0; q < E; ++q) {
            xk.v[q] = ys[(size_t)(k - s) * E + q];
            xk1.v[q] = ys[(size_t)(k - 1 - s) * E + q];
          }
          if (tid < 2 * E) pr.x[(size_t)(k - 1) * E + tid] = ys[(size_t)(k - 1 - s) * E + tid];
          const int t = tid;
          const bool act = t < 4 * (k - 1 - s);
          const int j = s + (t >> 2), part = (t >> 1) & 1, half = t & 1;
          double* yj = ys + (size_t)(act ? j - s : 0) * E;
          pacc a;
          Ar::pzero(a);
          if (act) {
            if (half == 0) Ar::pseed(a, yj + part * L);
            const int kk = half == 0 ? k : k - 1;
            const elem c = sm_load<Ar>(tb + ((size_t)(kk - s) * kBS + (j - s)) * E, 1, 0);
            elem xv;
#pragma unroll
            for (int q = 0; q < E; ++q) xv.v[q] = half == 0 ? xk.v[q] : xk1.v[q];
            Ar::mul_sub_half(f, a, c, xv, part, 0);
            Ar::mul_sub_half(f, a, c, xv, part, 1);
          }
          pacc o;
          const double* sa = reinterpret_cast<const double*>(&a);
          double* so = reinterpret_cast<double*>(&o);
#pragma unroll
          for (int q = 0; q < PACC; ++q) so[q] = __shfl_xor_sync(0xffffffffu, sa[q], 1);
          if (act && half == 0) {
            Ar::pcombine(f, a, o);
            Ar::pfinal(f, a, yj + part * L);
          }
          __syncthreads();
        }
        if ((nbk & 1) && tid < E) pr.x[(size_t)s * E + tid] = ys[tid];  // an odd block's last unknown
      } else {
        for (int k = e - 1; k >= s; --k) {
          elem xk;
#pragma unroll
          for (int q = 0; q < E; ++q) xk.v[q] = ys[(size_t)(k - s) * E + q];  // x~_k = y_k
          if (tid < E) pr.x[(size_t)k * E + tid] = ys[(size_t)(k - s) * E + tid];
          for (int t = tid; t < 2 * (k - s); t += T) {
            const int j = s + (t >> 1), part = t & 1;
            double* yj = ys + (size_t)(j - s) * E;
            elem y = sm_load_part<Ar>(yj, 1, 0, part);
            Ar::update_part(f, y, sm_load<Ar>(tb + ((size_t)(k - s) * kBS + (j - s)) * E, 1, 0), xk, part);
#pragma unroll
            for (int q = 0; q < L; ++q) yj[part * L + q] = y.v[part * L + q];
          }
          __syncthreads();
        }
      }
    }
    if (s == 0) break;
    grid_barrier(pr, epoch);
    // rows j < s: y_j -= sum_{k in [s, e)} t_jk x~_k; G lanes per (row, part) each sum a
    // share of the terms, a shuffle tree combines them, lane 0 of the group subtracts.  G is
    // the largest of 32, 16, 8 whose lanes the grid holds in one pass (fewest products per
    // lane), else 8.
    {
      int G = 32;
      while (G > 8 && s * 2 * G > nthreads) G >>= 1;
      const int tot = s * 2 * G;
      const int span = ((tot + nthreads - 1) / nthreads) * nthreads;  // uniform trip count
      for (int idx = gtid; idx < span; idx += nthreads) {
        const bool act = idx < tot;
        const int grp = idx / G, ch = idx % G;
        const int j = grp >> 1, part = grp & 1;
        pacc a;
        Ar::pzero(a);
        if (act)
          for (int k = e - 1 - ch; k >= s; k -= G)
            Ar::mul_acc_part(f, a, g_load_cg<Ar>(pr.Rt + ((size_t)k * n + j) * E),
                             g_load_cg<Ar>(pr.x + (size_t)k * E), part);
        for (int off = 1; off < G; off <<= 1) {
          pacc o;
          const double* sa = reinterpret_cast<const double*>(&a);
          double* so = reinterpret_cast<double*>(&o);
#pragma unroll
          for (int q = 0; q < PACC; ++q) so[q] = __shfl_xor_sync(0xffffffffu, sa[q], off);
          Ar::pcombine(f, a, o);
        }
        if (act && ch == 0) {
          double y[L];
          double* yp = pr.Y + (size_t)j * E + part * L;
#pragma unroll
          for (int q = 0; q < L; ++q) y[q] = __ldcg(yp + q);
          Ar::psub(f, y, a);
#pragma unroll
          for (int q = 0; q < L; ++q) yp[q] = y[q];
        }
      }
    }
    grid_barrier(pr, epoch);
  }
  grid_barrier(pr, epoch);
  // x_k = x~_k / r_kk
  for (int idx = gtid; idx < 2 * n; idx += nthreads) {
    const int k = idx >> 1, part = idx & 1;
    elem xt;
#pragma unroll
    for (int q = 0; q < E; ++q) xt.v[q] = 0.0;
#pragma unroll
    for (int q = 0; q < L; ++q) xt.v[part * L + q] = __ldcg(pr.x + (size_t)k * E + part * L + q);
    const real r = ld_real(pr.Rd + (size_t)k * L);
    elem xv = xt;
    Ar::div_real_part(f, xv, xt, r, Ar::inv_lead(r), part);
#pragma unroll
    for (int q = 0; q < L; ++q) pr.x[(size_t)k * E + part * L + q] = xv.v[part * L + q];
  }
  MGS_TR(nc, 3);
}

// ------------------------------------------------------------------ the kernel
template <class Ar, int T>
__global__ void __launch_bounds__(T, 1) mgs_ls_kernel(Params pr) {
  constexpr int L = Ar::L, E = 2 * L, ACC = Ar::ACC;
  using elem = typename Ar::elem;
  using acc = typename Ar::acc;
  using real = typename Ar::real;
  const Fp f{pr.one, pr.nzero};
  const int tid = threadIdx.x;
  const int Bc = pr.Bc, Br = pr.Br, nc = pr.nc, h = pr.h;
  const int p = blockIdx.x / Bc, c = blockIdx.x % Bc;
  const int r0 = p * h;
  const int hr = max(0, min(h, pr.m - r0));  // rows of this block that exist
  const int w = (nc - c + Bc - 1) / Bc;      // columns owned (slots)
  unsigned epoch = 0;

  extern __shared__ __align__(16) double sm[];
  double* tile = sm;                         // w * E * h
  double* piv = tile + (size_t)w * E * h;    // 2 * E * h
  double* coef = piv + (size_t)2 * E * h;    // w * E
  double* gkk = coef + (size_t)w * E;        // E (pivot norm, as an element)
  double* scal = gkk + E;                    // 4 * E scratch
  double* redb = scal + 4 * E;               // T part accumulators
  int* iflag = reinterpret_cast<int*>(redb + (size_t)T * L);
  using pacc = typename Ar::pacc;
  constexpr int PACC = Ar::PACC;
  static_assert(sizeof(pacc) == PACC * sizeof(double) && PACC == L, "part accumulator layout");

  auto col_of = [&](int s) { return c + s * Bc; };
  auto colptr = [&](int j, int i) -> double* {
    return (j < pr.n) ? pr.A + ((size_t)j * pr.lda + i) * E : pr.b + (size_t)i * E;
  };
  auto ld_real = [&](const double* src) {
    real r;
    double* d = reinterpret_cast<double*>(&r);
#pragma unroll
    for (int q = 0; q < L; ++q) d[q] = __ldcg(src + q);
    return r;
  };
  auto st_real = [&](double* dst, const real& r) {
    const double* d = reinterpret_cast<const double*>(&r);
#pragma unroll
    for (int q = 0; q < L; ++q) dst[q] = d[q];
  };

  if (pr.skip && *pr.skip) return;  // uniform over the grid: no barrier is entered
  MGS_TR_SMID();
  // ---------------------------------------------------------------- load the tile
  if (tid == 0) iflag[0] = 0;
  __syncthreads();
  {
    bool bad = false;
    for (int idx = tid; idx < w * h; idx += T) {
      const int s = idx / h, l = idx % h;
      elem e;
      if (l < hr) {
        e = g_load<Ar>(colptr(col_of(s), r0 + l));
#pragma unroll
        for (int q = 0; q < E; ++q) bad |= !finite64(e.v[q]);
      } else {
#pragma unroll
        for (int q = 0; q < E; ++q) e.v[q] = 0.0;
      }
      sm_store<Ar>(tile + (size_t)s * E * h, h, l, e);
    }
    if (bad) iflag[0] = 1;
  }
  // pivot 0 rows (column 0 is unmodified at the start)
  for (int l = tid; l < h; l += T) {
    elem e;
    if (l < hr) {
      e = g_load<Ar>(colptr(0, r0 + l));
    } else {
#pragma unroll
      for (int q = 0; q < E; ++q) e.v[q] = 0.0;
    }
    sm_store<Ar>(piv, h, l, e);
  }
  __syncthreads();
  if (tid == 0 && iflag[0]) set_status(pr.status, ST_ENONFINITE);

  // Partials of the Gram row of pivot `kp` (pivot rows in pivbuf) for own columns j >= kp,
  // written to P[buf].  Work items are (column, part, row chunk): all lanes get about the
  // same number of rows; the chunks of one (column, part) are combined by a tree in
  // shared memory.  For the pivot column only the real part (its norm) is formed.
  auto partials = [&](int kp, const double* pivbuf, int buf) {
    const int s0 = (kp - c + Bc - 1) / Bc;  // first slot with column >= kp
    const int first = max(s0, 0);
    const int nact = w - first;
    if (nact <= 0) return;
    const int pairs = 2 * nact;
    int C = T / pairs;
    C = max(1, min(C, max(hr, 1)));
    const int per_round = T / C;
    pacc* red = reinterpret_cast<pacc*>(redb);
    if (flat_partials_cheaper<Ar, T>(pairs, hr, C)) {
      // Flat mapping: the pairs * hr (pair, row) items in order, `per` consecutive items per
      // lane, so every lane does the same number of products.  A lane whose items run
      // into the next pair keeps a second accumulator (in the coefficient area, dead
      // during the partials).  The lanes starting in one pair combine by a tree rooted at
      // the first of them, which then folds in the second accumulator of the lane before.
      const int items = pairs * hr;
      const int per = (items + T - 1) / T;
      const int lev = ceil_log2((hr + per - 1) / per);
      pacc* carry = reinterpret_cast<pacc*>(coef);  // one slot per pair (w E doubles = 2w pacc)
      const int st = tid * per, en = min(st + per, items);
      const bool act = st < items;
      const int p0 = act ? st / hr : 0;
      const int fl = (p0 * hr + per - 1) / per;                   // first lane starting in pair p0
      const int cnt = (min((p0 + 1) * hr, items) - 1) / per - fl + 1;  // lanes starting in pair p0
      // One loop of `per` iterations for every lane (two loops, one per pair, would run one
      // after the other in a warp that holds a lane crossing a pair boundary).  The pivot
      // column's imaginary part is computed like any other and written as zero.
      const int bnd = min(en, (p0 + 1) * hr);
      const bool cross = act && en > bnd;  // this lane's items run into pair p0 + 1
      pacc a, cur;
      Ar::pzero(a);
      Ar::pzero(cur);
      for (int it = 0; it < per; ++it) {
        const int i = st + it;
        if (cross && i == bnd) {  // keep the first pair's sum, start the second
          a = cur;
          Ar::pzero(cur);
        }
        const int pp = i < bnd ? p0 : p0 + 1;
        const int s = first + (pp >> 1), part = pp & 1, l = i - pp * hr;
        if (i < en) Ar::mac_part(f, cur, sm_load<Ar>(pivbuf, h, l), sm_load<Ar>(tile + (size_t)s * E * h, h, l), part);
      }
      if (cross) {
        carry[p0 + 1] = cur;
      } else {
        a = cur;
      }
      red[tid] = a;
      __syncthreads();
      const int idx = tid - fl;
      for (int stp = 1; stp < (1 << lev); stp <<= 1) {
        if (act && (idx % (2 * stp)) == 0 && idx + stp < cnt) {
          pacc x = red[tid];
          Ar::pcombine(f, x, red[tid + stp]);
          red[tid] = x;
        }
        __syncthreads();
      }
      if (act && idx == 0) {
        pacc x = red[tid];
        if (st != p0 * hr) Ar::pcombine(f, x, carry[p0]);  // lane tid - 1 ran into this pair
        const int j = col_of(first + (p0 >> 1));
        if (j == kp && (p0 & 1)) Ar::pzero(x);
        const double* src = reinterpret_cast<const double*>(&x);
        double* dst = pr.P + (((size_t)buf * Br + p) * nc + j) * ACC + (p0 & 1) * PACC;
#pragma unroll
        for (int q = 0; q < PACC; ++q) dst[q] = src[q];
      }
      __syncthreads();
      return;
    }
    for (int base = 0; base < pairs; base += per_round) {
      const int job = tid / C, ch = tid % C;
      const int pi = base + job;
      const bool act = job < per_round && pi < pairs;
      const int s = first + (pi >> 1), part = pi & 1;
      pacc a;
      Ar::pzero(a);
      if (act) {
        const int j = col_of(s);
        if (!(j == kp && part == 1)) {
          const double* ts = tile + (size_t)s * E * h;
          for (int l = ch; l < hr; l += C) Ar::mac_part(f, a, sm_load<Ar>(pivbuf, h, l), sm_load<Ar>(ts, h, l), part);
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
        const int j = col_of(s);
        const double* src = reinterpret_cast<const double*>(&red[tid]);
        double* dst = pr.P + (((size_t)buf * Br + p) * nc + j) * ACC + part * PACC;
#pragma unroll
        for (int q = 0; q < PACC; ++q) dst[q] = src[q];
      }
      __syncthreads();
    }
  };

  partials(0, piv, 0);
  grid_barrier(pr, epoch);

  // ---------------------------------------------------------------- the steps
  for (int k = 0; k < nc; ++k) {
    const int cur = k & 1, nxt = cur ^ 1;
    const double* pcur = piv + (size_t)cur * E * h;
    double* pnxt = piv + (size_t)nxt * E * h;
    const bool own_k = (k % Bc) == c;
    const bool last = (k == nc - 1);
    const bool own_k1 = !last && ((k + 1) % Bc) == c;
    const int s0 = (k + 1 - c + Bc - 1) / Bc;  // first slot with column > k
    const int first = max(s0, 0);
    const int nact = w - first;                // own columns j > k
    MGS_TR(k, 0);

    // (1) reduce the Br partials of the pivot norm and of the own columns j > k: g lanes
    //     per (column, part), lane pp folding row blocks pp, pp + g, ..., then a shuffle
    //     tree over the g lanes.  g is the largest power of two up to Br that fits the busiest
    //     CTA's jobs in one round, the same in every CTA, so G_kk is summed in the same
    //     order everywhere.
    {
      const int BrP = pow2_ceil(Br);
      const int nred = 1 + max(nact, 0);
      const int nact_max = (nc - 1 - k + Bc - 1) / Bc;
      int g = BrP;
      while (g > 1 && (1 + nact_max) * 2 * g > T) g >>= 1;
      const int jobs = nred * 2 * g;
      for (int base = 0; base < jobs; base += T) {
        const int job = base + tid;
        const int ci = job / (2 * g), rem = job % (2 * g);
        const int part = rem / g, pp = rem % g;
        const bool want = job < jobs && !(ci == 0 && part == 1);
        pacc a;
        Ar::pzero(a);
        if (want && pp < Br) {
          const int j = (ci == 0) ? k : col_of(first + ci - 1);
          double* d = reinterpret_cast<double*>(&a);
#pragma unroll
          for (int q = 0; q < PACC; ++q) d[q] = __ldcg(pr.P + (((size_t)cur * Br + pp) * nc + j) * ACC + part * PACC + q);
          for (int qb = pp + g; qb < Br; qb += g) {
            pacc o;
            double* od = reinterpret_cast<double*>(&o);
#pragma unroll
            for (int q = 0; q < PACC; ++q) od[q] = __ldcg(pr.P + (((size_t)cur * Br + qb) * nc + j) * ACC + part * PACC + q);
            Ar::pcombine(f, a, o);
          }
        }
        for (int off = 1; off < g; off <<= 1) {
          pacc o;
          const double* sa = reinterpret_cast<const double*>(&a);
          double* so = reinterpret_cast<double*>(&o);
#pragma unroll
          for (int q = 0; q < PACC; ++q) so[q] = __shfl_xor_sync(0xffffffffu, sa[q], off);
          Ar::pcombine(f, a, o);
        }
        if (job < jobs && pp == 0) {
          double* dst = ((ci == 0) ? gkk : coef + (size_t)(first + ci - 1) * E) + part * L;
          if (want) {
            Ar::pfinal(f, a, dst);
          } else {
#pragma unroll
            for (int q = 0; q < L; ++q) dst[q] = 0.0;
          }
        }
      }
    }
    __syncthreads();
    MGS_TR(k, 1);
    // pivot norm G_kk (identical in every CTA)
    elem gk;
#pragma unroll
    for (int q = 0; q < E; ++q) gk.v[q] = gkk[q];
    const real G = Ar::re(gk);
    const bool okpiv = Ar::positive(G);
    if (blockIdx.x == 0 && tid == 0) {
      st_real(pr.Gd + (size_t)k * L, G);
      if (!okpiv && !(last && pr.aug)) set_status(pr.status, ST_ERANK);
    }

    if (last && pr.aug) {
      // the right-hand-side column: what is left of it is the residual b - A x
      if (own_k) {
        const int s = k / Bc;
        const double* ts = tile + (size_t)s * E * h;
        for (int l = tid; l < hr; l += T) g_store<Ar>(pr.b + (size_t)(r0 + l) * E, sm_load<Ar>(ts, h, l));
      }
      break;
    }

    // (2) coefficients c_kj = G_kj / G_kk of the own columns j > k, one lane per part
    {
      const double invG = Ar::inv_lead(G);
      for (int t = tid; t < 2 * nact; t += T) {
        double* cs = coef + (size_t)(first + (t >> 1)) * E;
        const int part = t & 1;
        const elem g = sm_load_part<Ar>(cs, 1, 0, part);
        elem cc = g;
        if (okpiv) {
          Ar::div_real_part(f, cc, g, G, invG, part);
        } else {
#pragma unroll
          for (int q = 0; q < E; ++q) cc.v[q] = 0.0;
        }
#pragma unroll
        for (int q = 0; q < L; ++q) cs[part * L + q] = cc.v[part * L + q];
      }
    }
    __syncthreads();

    MGS_TR(k, 2);
    // (3) look-ahead: update column k+1 first and publish its rows
    if (own_k1) {
      const int s1 = (k + 1) / Bc;
      double* ts = tile + (size_t)s1 * E * h;
      elem cc;
#pragma unroll
      for (int q = 0; q < E; ++q) cc.v[q] = coef[(size_t)s1 * E + q];
      for (int t = tid; t < 2 * hr; t += T) {
        const int l = t >> 1, part = t & 1;
        elem y = sm_load_part<Ar>(ts, h, l, part);
        Ar::update_part(f, y, cc, sm_load<Ar>(pcur, h, l), part);
#pragma unroll
        for (int q = 0; q < L; ++q) {
          ts[(part * L + q) * h + l] = y.v[part * L + q];
          pnxt[(part * L + q) * h + l] = y.v[part * L + q];
        }
      }
      for (int l = hr + tid; l < h; l += T) {  // padding rows stay zero
#pragma unroll
        for (int q = 0; q < E; ++q) pnxt[q * h + l] = 0.0;
      }
      __syncthreads();
      double* vdst = pr.V + ((size_t)nxt * Br + p) * h * E;
      for (int l = tid; l < h; l += T) g_store<Ar>(vdst + (size_t)l * E, sm_load<Ar>(pnxt, h, l));
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        st_release_s32(pr.flags + (size_t)(k + 1) * Br + p, 1);
      }
    }

    MGS_TR(k, 3);
    // (4) update the other own columns j > k+1.  A CTA that does not own column k+1 reads
    //     the pivot-ready flag before its second-to-last column (by then the owners, who
    //     updated column k+1 first, have usually published it) and, when it was set, loads
    //     its row of the new pivot into registers before the last column: the two memory
    //     latencies of step (6) then pass under the updates.  Each thread takes the flag
    //     with its own acquire load, which orders its reads of the pivot rows.
    const int* flag1 = pr.flags + (size_t)(k + 1) * Br + p;
    const double* vsrc = pr.V + ((size_t)nxt * Br + p) * h * E;
    bool have = false;  // this thread's pivot row (row tid when tid < h) is in pv
    elem pv;
    {
      const int sb = own_k1 ? first + 1 : first;  // slot of column k+1 is `first` when owned
      const int nb = w - sb;
      if (!own_k1 && !last && nb >= 3 && T >= h) {
        update_slots<Ar, T>(f, tile, coef, pcur, h, hr, sb, nb - 2);
        const int fv = ld_acquire_s32(flag1);  // first used after the next column
        update_slots<Ar, T>(f, tile, coef, pcur, h, hr, sb + nb - 2, 1);
        if (fv != 0) {
          if (tid < h) pv = g_load_cg<Ar>(vsrc + (size_t)tid * E);
          have = true;
        }
        update_slots<Ar, T>(f, tile, coef, pcur, h, hr, sb + nb - 1, 1);
      } else {
        update_slots<Ar, T>(f, tile, coef, pcur, h, hr, sb, nb);
      }
    }

    MGS_TR(k, 4);
    // (5) coefficients of row k go to R (row k) and Y (column b); scaled by r_kk at the end
    if (p == 0) {
      for (int t = tid; t < nact; t += T) {
        const int s = first + t, j = col_of(s);
        elem cc;
#pragma unroll
        for (int q = 0; q < E; ++q) cc.v[q] = coef[(size_t)s * E + q];
        if (j < pr.n)
          g_store<Ar>(pr.R + ((size_t)j * pr.ldr + k) * E, cc);
        else
          g_store<Ar>(pr.Y + (size_t)k * E, cc);
      }
    }

    if (last) break;  // plain QR: every column has been reduced

    // (6) the new pivot rows for the CTAs that do not own column k+1 (prefetched in (4)
    //     when every thread saw the flag set)
    if (!own_k1) {
      if (__syncthreads_and(have)) {
        if (tid < h) sm_store<Ar>(pnxt, h, tid, pv);
      } else {
        if (tid == 0) wait_flag(pr, flag1);
        __syncthreads();
        for (int l = tid; l < h; l += T) sm_store<Ar>(pnxt, h, l, g_load_cg<Ar>(vsrc + (size_t)l * E));
      }
    }
    __syncthreads();

    MGS_TR(k, 5);
    // (7) partials of step k+1
    partials(k + 1, pnxt, nxt);
    MGS_TR(k, 6);
    grid_barrier(pr, epoch);
  }
  grid_barrier(pr, epoch);
  MGS_TR(nc, 0);

  mgs_epilogue<Ar, T>(pr, epoch, sm, p, c);
}

}  // namespace mgs
