// Single-system MGS least squares without a grid-wide barrier per step: the Br CTAs that
// own the rows of one column group form a thread-block cluster and reduce their Gram
// partials through distributed shared memory; the pivots travel between clusters through
// release/acquire flags.  Same method, tiles and arithmetic as mgs_ls_kernel (Section 3,
// Figure 1 and Eq. 1; Section 6, Figure 3).
//
// The pivot hand-off chain (the critical path): the cluster that owns column k+1 turns it
// into pivot k+1 in step k (A: partials of G_kk = ||a_k||^2 and G_{k,k+1} over its rows ->
// cluster reduction -> c_{k,k+1} = G_{k,k+1} / G_kk -> update column k+1 -> publish its
// rows).  Two-step look-ahead: the cluster that owns column k+2 applies pivot k to that
// column first (the same phase without the publication), then waits for pivot k+1 and runs
// A(k+1) at once, and only then does its bulk work of steps k and k+1.  So no cluster does
// bulk work between receiving the pivot before its own and publishing its own, and the
// chain advances at the speed of A plus the hand-off, not of the bulk.
//   Bulk (B) of step k in every cluster: partials of its other trailing columns (and of
//   G_kk where no critical phase formed it) -> cluster reduction -> coefficients ->
//   update -> (wait for the rows of pivot k+1).
// Every cluster forms G_kk from the pivot rows it holds, so nothing but the pivot itself
// passes between clusters.  The clusters sum G_kk's terms in different orders; the owner of
// column k+1 stores its value, which gives r_kk.  One grid barrier before the
// normalisation epilogue.
//
// HW = true: the Br CTAs form a hardware cluster (cluster.sync, partials read through
// distributed shared memory); clusters must fit in a GPC, which can leave SMs idle.
// HW = false: the same schedule on a plain cooperative grid; the Br CTAs meet at a
// counter in global memory and exchange their partials through L2, so every SM can
// hold a CTA.
#pragma once

#include <cooperative_groups.h>

#include "mgs_kernel.cuh"

namespace mgs {

// Barrier of the Br CTAs of one column group on a monotone arrival counter in global
// memory (bounded like grid_barrier: gives up on the abort flag or after the time limit).
__device__ __forceinline__ void group_barrier(const Params& pr, unsigned* ctr, unsigned& gepoch, int members) {
  __syncthreads();
  if (threadIdx.x == 0) {
    ++gepoch;
    const unsigned target = gepoch * (unsigned)members;
    __threadfence();
    const unsigned arrived = atomicAdd(ctr, 1u) + 1u;
    if (arrived < target) {  // the last member to arrive does not poll
      const unsigned long long t0 = globaltimer();
      unsigned spins = 0;
      while (ld_acquire_u32(ctr) < target) {
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

// Doubles of global partials the HW = false variant needs (two B buffers and two A
// buffers per CTA, `wmax` = columns of the widest group).
__host__ __device__ inline size_t group_partials_doubles(int L, int Br, int Bc, int wmax) {
  return (size_t)Bc * Br * (2 * (size_t)(wmax + 1) * 2 * L + (size_t)2 * 2 * 2 * L);
}

// Shared memory of the cluster kernel: the tile and three pivot buffers (pivots k, k+1
// and k+2 are live at once in the look-ahead), coefficients, scalars, the reduction tree,
// B partials (two buffers of w + 1 items x 2 parts), A partials (two buffers of 2 items x
// 2 parts), reduced values.
__host__ __device__ inline size_t cluster_smem_bytes(int L, int h, int w, int T) {
  return smem_bytes(L, h, w, T) + sizeof(double) * ((size_t)2 * L * h + 2 * (size_t)(w + 1) * 2 * L +
                                                    (size_t)2 * 2 * 2 * L + (size_t)(w + 2) * 2 * L) +
         64;
}

template <class Ar, bool HW, int T>
__global__ void __launch_bounds__(T, 1) mgs_cluster_kernel(Params pr) {
  namespace cg = cooperative_groups;
  constexpr int L = Ar::L, E = 2 * L;
  using elem = typename Ar::elem;
  using real = typename Ar::real;
  using pacc = typename Ar::pacc;
  constexpr int PACC = Ar::PACC;
  static_assert(sizeof(pacc) == PACC * sizeof(double) && PACC == L, "part accumulator layout");
  cg::cluster_group cluster = cg::this_cluster();
  const Fp f{pr.one, pr.nzero};
  const int tid = threadIdx.x;
  const int Bc = pr.Bc, Br = pr.Br, nc = pr.nc, h = pr.h;
  const int p = HW ? (int)cluster.block_rank() : (int)(blockIdx.x % Br);
  const int c = blockIdx.x / Br;
  const int r0 = p * h;
  const int hr = max(0, min(h, pr.m - r0));
  const int w = (nc - c + Bc - 1) / Bc;
  // published pivot rows live in a ring of Bc + 2 slots.  A cluster loads every pivot below
  // a column before it publishes that column (it takes the steps in order, and the
  // look-ahead only moves its bulk work later); every cluster that still has work after
  // step j owns one of the columns j + 1 .. j + Bc; and pivots are published in order (each
  // owner waits for the previous pivot).  So by the time pivot j + Bc + 1 or later is
  // written, every cluster that needs pivot j has loaded it, and slot j is free again.
  const int vslots = Bc + 2;
  unsigned epoch = 0, gepoch = 0;
  unsigned* gctr = pr.gsync + (size_t)c * 32;  // this group's arrival counter (HW = false)
  auto group_sync = [&]() {
    if constexpr (HW)
      cluster.sync();
    else
      group_barrier(pr, gctr, gepoch, Br);
  };

  extern __shared__ __align__(16) double sm[];
  double* tile = sm;                         // w * E * h
  double* piv = tile + (size_t)w * E * h;    // 3 * E * h: pivot k in buffer k % 3
  double* coef = piv + (size_t)3 * E * h;    // w * E
  double* gkk = coef + (size_t)w * E;        // E
  double* scal = gkk + E;                    // 4 * E
  double* redb = scal + 4 * E;               // T * L
  double* pbuf = redb + (size_t)T * L;        // 2 x (w + 1) x 2 x PACC
  double* pabuf = pbuf + 2 * (size_t)(w + 1) * 2 * PACC;  // 2 x 2 x 2 x PACC
  double* gres = pabuf + 2 * 2 * 2 * PACC;           // (w + 2) x E reduced values
  // HW = false: the partial buffers live in global memory, CTA-major within a group so
  // that peer pp's buffer is `stride` doubles from ours
  const int wmax = (nc + Bc - 1) / Bc;
  const size_t gstride = 2 * (size_t)(wmax + 1) * 2 * PACC + (size_t)2 * 2 * 2 * PACC;
  if constexpr (!HW) {
    pbuf = pr.P + ((size_t)c * Br + p) * gstride;
    pabuf = pbuf + 2 * (size_t)(wmax + 1) * 2 * PACC;
  }
  const int pbw = HW ? w : wmax;  // B-buffer width in items - 1
  int* iflag = reinterpret_cast<int*>(gres + (size_t)(w + 2) * E);
  pacc* red = reinterpret_cast<pacc*>(redb);
  (void)scal;
  (void)gkk;
  auto pbk = [&](int k) { return piv + (size_t)(k % 3) * E * h; };  // pivot k's rows

  auto col_of = [&](int s) { return c + s * Bc; };
  auto colptr = [&](int j, int i) -> double* {
    return (j < pr.n) ? pr.A + ((size_t)j * pr.lda + i) * E : pr.b + (size_t)i * E;
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

  // Partials over this CTA's rows of the items it = 0..nit-1: item -> slot (or -1: the
  // pivot's norm, real part only).  (item, part, row chunk) work items; tree in shared
  // memory; results at out[(it * 2 + part) * PACC].
  auto item_partials = [&](const double* pivbuf, int nit, auto slot_of, double* out) {
    const int pairs = 2 * nit;
    int C = T / pairs;
    C = max(1, min(C, max(hr, 1)));
    const int per_round = T / C;
    for (int base = 0; base < pairs; base += per_round) {
      const int job = tid / C, ch = tid % C, pi = base + job;
      const bool act = job < per_round && pi < pairs;
      const int it = pi >> 1, part = pi & 1;
      const int s = act ? slot_of(it) : 0;
      pacc a;
      Ar::pzero(a);
      if (act && !(s < 0 && part == 1)) {
        const double* ts = (s < 0) ? pivbuf : tile + (size_t)s * E * h;
        for (int l = ch; l < hr; l += C) Ar::mac_part(f, a, sm_load<Ar>(pivbuf, h, l), sm_load<Ar>(ts, h, l), part);
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
        const double* src = reinterpret_cast<const double*>(&red[tid]);
#pragma unroll
        for (int q = 0; q < PACC; ++q) out[(size_t)pi * PACC + q] = src[q];
      }
      __syncthreads();
    }
  };

  // Sum over the cluster's Br CTAs of the partials in `buf` (nit items): one lane per
  // (item, part, peer), read through distributed shared memory, shuffle tree; results
  // into gres (item it at it * E).  The pivot-norm item has no imaginary part.
  auto cluster_reduce = [&](double* buf, int nit, auto is_norm) {
    const int BrP = pow2_ceil(Br);
    const int jobs = nit * 2 * BrP;
    for (int base = 0; base < jobs; base += T) {
      const int job = base + tid;
      const int it = job / (2 * BrP), rem = job % (2 * BrP);
      const int part = rem / BrP, pp = rem % BrP;
      const bool want = job < jobs && !(is_norm(it) && part == 1);
      pacc a;
      Ar::pzero(a);
      if (want && pp < Br) {
        double* d = reinterpret_cast<double*>(&a);
        if constexpr (HW) {
          const double* peer = cluster.map_shared_rank(buf, pp);
#pragma unroll
          for (int q = 0; q < PACC; ++q) d[q] = peer[((size_t)it * 2 + part) * PACC + q];
        } else {
          const double* peer = buf + ((long long)pp - p) * (long long)gstride;
#pragma unroll
          for (int q = 0; q < PACC; ++q) d[q] = __ldcg(peer + ((size_t)it * 2 + part) * PACC + q);
        }
      }
      for (int off = 1; off < BrP; off <<= 1) {
        pacc o;
        const double* sa = reinterpret_cast<const double*>(&a);
        double* so = reinterpret_cast<double*>(&o);
#pragma unroll
        for (int q = 0; q < PACC; ++q) so[q] = __shfl_xor_sync(0xffffffffu, sa[q], off);
        Ar::pcombine(f, a, o);
      }
      if (job < jobs && pp == 0) {
        double* dst = gres + (size_t)it * E + part * L;
        if (want) {
          Ar::pfinal(f, a, dst);
        } else {
#pragma unroll
          for (int q = 0; q < L; ++q) dst[q] = 0.0;
        }
      }
    }
    __syncthreads();
  };

  auto coef_of = [&](int s, const real& G, bool ok, const double* gsrc) {
    const double invG = Ar::inv_lead(G);
    for (int t = tid; t < 2; t += T) {
      const int part = t;
      const elem g = sm_load_part<Ar>(gsrc, 1, 0, part);
      elem cc = g;
      if (ok) {
        Ar::div_real_part(f, cc, g, G, invG, part);
      } else {
#pragma unroll
        for (int q = 0; q < E; ++q) cc.v[q] = 0.0;
      }
#pragma unroll
      for (int q = 0; q < L; ++q) coef[(size_t)s * E + part * L + q] = cc.v[part * L + q];
    }
  };

  unsigned bph = 0;  // B reductions so far (selects the B-partials buffer)

  // Critical phase: pivot kk (rows at pbk(kk)) applied to the owned column j alone --
  // partials of G_kk and G_{kk,j} over this CTA's rows, cluster reduction, c_{kk,j},
  // update of column j (row kk of R stored).  With `publish` (j = kk + 1) the updated
  // rows are pivot kk + 1: copied to pbk(kk + 1), published in the ring with this row
  // block's flag, and G_kk is recorded.  Returns G_kk.  `ab` selects the A-partials buffer
  // (the pre-phase and the phase that follows it use different ones).
  auto critical = [&](int kk, int j, bool publish, int ab) -> real {
    MGS_TR(kk, 1);
    const double* pc = pbk(kk);
    const int sj = (j - c) / Bc;
    double* pa = pabuf + (size_t)ab * 2 * 2 * PACC;
    item_partials(pc, 2, [&](int it) { return it == 0 ? -1 : sj; }, pa);
    group_sync();
    cluster_reduce(pa, 2, [](int it) { return it == 0; });
    const real G = Ar::re(sm_load<Ar>(gres, 1, 0));
    const bool ok = Ar::positive(G);
    if (publish && p == 0 && tid == 0) {
      st_real(pr.Gd + (size_t)kk * L, G);
      if (!ok) set_status(pr.status, ST_ERANK);
    }
    coef_of(sj, G, ok, gres + E);
    __syncthreads();
    double* ts = tile + (size_t)sj * E * h;
    elem cc;
#pragma unroll
    for (int q = 0; q < E; ++q) cc.v[q] = coef[(size_t)sj * E + q];
    if (p == 0 && tid == 0) g_store<Ar>(j < pr.n ? pr.R + ((size_t)j * pr.ldr + kk) * E : pr.Y + (size_t)kk * E, cc);
    double* pn = publish ? pbk(kk + 1) : nullptr;
    for (int t = tid; t < 2 * hr; t += T) {
      const int l = t >> 1, part = t & 1;
      elem y = sm_load_part<Ar>(ts, h, l, part);
      Ar::update_part(f, y, cc, sm_load<Ar>(pc, h, l), part);
#pragma unroll
      for (int q = 0; q < L; ++q) {
        ts[(part * L + q) * h + l] = y.v[part * L + q];
        if (publish) pn[(part * L + q) * h + l] = y.v[part * L + q];
      }
    }
    if (publish) {
      for (int l = hr + tid; l < h; l += T) {
#pragma unroll
        for (int q = 0; q < E; ++q) pn[q * h + l] = 0.0;
      }
      __syncthreads();
      double* vdst = pr.V + ((size_t)((kk + 1) % vslots) * Br + p) * h * E;
      for (int l = tid; l < h; l += T) g_store<Ar>(vdst + (size_t)l * E, sm_load<Ar>(pn, h, l));
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        st_release_s32(pr.flags + (size_t)(kk + 1) * Br + p, 1);
      }
    } else {
      __syncthreads();
    }
    MGS_TR(kk, 5);
    return G;
  };

  // Bulk phase of step kk on the owned slots [sb, w): partials (with G_kk's unless
  // `haveG`), cluster reduction, coefficients, R/y stores, updates.  Returns G_kk.
  auto bulk = [&](int kk, int sb, bool haveG, real G) -> real {
    MGS_TR(kk, 0);
    const double* pc = pbk(kk);
    const bool norm_here = !haveG;
    const int nb = w - sb;
    const int nitB = nb + (norm_here ? 1 : 0);
    if (nitB > 0) {
      // the two buffers alternate between consecutive reductions: a peer reads one while
      // this CTA may already write the other, and a buffer is written again only after
      // the next reduction's cluster barrier
      double* pb = pbuf + (size_t)(bph & 1u) * (pbw + 1) * 2 * PACC;
      ++bph;
      auto slotB = [&](int it) { return norm_here ? (it == 0 ? -1 : sb + it - 1) : sb + it; };
      item_partials(pc, nitB, slotB, pb);
      MGS_TR(kk, 6);
      group_sync();
      cluster_reduce(pb, nitB, [&](int it) { return norm_here && it == 0; });
    }
    MGS_TR(kk, 2);
    if (norm_here) G = Ar::re(sm_load<Ar>(gres, 1, 0));
    if (nb <= 0) return G;
    const bool okpiv = Ar::positive(G);
    {
      const double invG = Ar::inv_lead(G);
      const int ib = norm_here ? 1 : 0;
      for (int t = tid; t < 2 * nb; t += T) {
        const int it = t >> 1, part = t & 1, s = sb + it;
        const elem g = sm_load_part<Ar>(gres + (size_t)(it + ib) * E, 1, 0, part);
        elem cc = g;
        if (okpiv) {
          Ar::div_real_part(f, cc, g, G, invG, part);
        } else {
#pragma unroll
          for (int q = 0; q < E; ++q) cc.v[q] = 0.0;
        }
#pragma unroll
        for (int q = 0; q < L; ++q) coef[(size_t)s * E + part * L + q] = cc.v[part * L + q];
      }
    }
    __syncthreads();
    MGS_TR(kk, 3);
    // coefficients of row kk to R (row kk) and Y (column b); scaled by r_kk at the end
    if (p == 0) {
      for (int t = tid; t < nb; t += T) {
        const int s = sb + t, j = col_of(s);
        elem cc;
#pragma unroll
        for (int q = 0; q < E; ++q) cc.v[q] = coef[(size_t)s * E + q];
        if (j < pr.n)
          g_store<Ar>(pr.R + ((size_t)j * pr.ldr + kk) * E, cc);
        else
          g_store<Ar>(pr.Y + (size_t)kk * E, cc);
      }
    }
    update_slots<Ar, T>(f, tile, coef, pc, h, hr, sb, nb);
    __syncthreads();  // the next phase reads these columns (threads update other elements)
    MGS_TR(kk, 4);
    return G;
  };

  // the rows of pivot kk, published by its owner, into pbk(kk)
  auto receive = [&](int kk) {
    if (tid == 0) wait_flag(pr, pr.flags + (size_t)kk * Br + p);
    __syncthreads();
    const double* vsrc = pr.V + ((size_t)(kk % vslots) * Br + p) * h * E;
    double* dst = pbk(kk);
    for (int l = tid; l < h; l += T) sm_store<Ar>(dst, h, l, g_load_cg<Ar>(vsrc + (size_t)l * E));
    __syncthreads();
    MGS_TR(kk, 7);  // kk >= 1: slot 7 of step 0 holds the SM id
  };

  // ---------------------------------------------------------------- the steps
  for (int k = 0; k < nc;) {
    const bool last = (k == nc - 1);
    const bool own_k = (k % Bc) == c;
    const bool own_k1 = !last && ((k + 1) % Bc) == c;
    const bool own_k2 = Bc >= 2 && k + 2 < nc && ((k + 2) % Bc) == c;  // then !own_k1
    const int s0 = (k + 1 - c + Bc - 1) / Bc;
    const int first = max(s0, 0);  // first owned slot with a column > k
    const int nact = w - first;    // owned columns j > k
    if (nact <= 0 && !(last && own_k)) break;  // nothing left for this cluster

    if (own_k2) {
      // column k+2 is the next pivot this cluster publishes: pivot k, then pivot k+1 on it
      // before any bulk work; the bulk of steps k and k+1 follows
      const real G0 = critical(k, k + 2, false, 0);
      receive(k + 1);
      const real G1 = critical(k + 1, k + 2, true, 1);
      bulk(k, first + 1, true, G0);
      bulk(k + 1, first + 1, true, G1);
      k += 2;  // pivot k+2 is this cluster's own, already in pbk(k + 2)
      continue;
    }

    real G{};
    if (own_k1) G = critical(k, k + 1, true, 1);
    G = bulk(k, own_k1 ? first + 1 : first, own_k1, G);
    if (last) {
      // only the owner of the last column is left; for [A b] its norm is z and what is
      // left of it is the residual b - A x
      if (p == 0 && tid == 0) {
        st_real(pr.Gd + (size_t)k * L, G);
        if (!pr.aug && !Ar::positive(G)) set_status(pr.status, ST_ERANK);
      }
      if (pr.aug) {
        const double* ts = tile + (size_t)(k / Bc) * E * h;
        for (int l = tid; l < hr; l += T) g_store<Ar>(pr.b + (size_t)(r0 + l) * E, sm_load<Ar>(ts, h, l));
      }
      break;
    }
    // the rows of pivot k+1
    if (!own_k1) receive(k + 1);
    ++k;
  }
  // no CTA may go on (and, after an abort, exit) while a peer still reads its shared
  // memory; then the epilogue needs all columns, rows of R and G_kk
  group_sync();
  grid_barrier(pr, epoch);
  MGS_TR(nc, 0);
  mgs_epilogue<Ar, T>(pr, epoch, sm, p, c);
}

}  // namespace mgs
