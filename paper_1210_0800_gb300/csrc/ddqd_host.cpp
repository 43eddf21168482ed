// Host build of the device DD/QD arithmetic (ddqd.cuh compiled as plain C++) so the test
// suite can check the exact operations the kernels perform against exact rationals on
// the CPU.  The host intrinsics are correctly rounded like the GPU's, so the results are
// the same bits.  Not used by the solver itself.
#include "ddqd.cuh"

namespace {

const mgs::Fp kFp{1.0, -0.0};

template <class Ar>
typename Ar::elem load(const double* p) {
  typename Ar::elem e;
  for (int q = 0; q < 2 * Ar::L; ++q) e.v[q] = p[q];
  return e;
}
template <class Ar>
void store(double* p, const typename Ar::elem& e) {
  for (int q = 0; q < 2 * Ar::L; ++q) p[q] = e.v[q];
}
template <class Ar>
typename Ar::real load_real(const double* p) {
  typename Ar::real r;
  double* d = reinterpret_cast<double*>(&r);
  for (int q = 0; q < Ar::L; ++q) d[q] = p[q];
  return r;
}
template <class Ar>
void store_real(double* p, const typename Ar::real& r) {
  const double* d = reinterpret_cast<const double*>(&r);
  for (int q = 0; q < Ar::L; ++q) p[q] = d[q];
}

template <class Ar>
void dot(int n, int split, const double* x, const double* y, double* out, bool norm) {
  const int E = 2 * Ar::L;
  typename Ar::acc a, b;
  Ar::zero(a);
  Ar::zero(b);
  for (int i = 0; i < n; ++i) {
    auto& t = (i < split) ? a : b;
    if (norm)
      Ar::mac_norm(kFp, t, load<Ar>(x + i * E));
    else
      Ar::mac_conj(kFp, t, load<Ar>(x + i * E), load<Ar>(y + i * E));
  }
  Ar::combine(kFp, a, b);
  store<Ar>(out, Ar::finalize(kFp, a));
}

template <class Ar>
void dot_parts(int n, int split, const double* x, const double* y, double* out) {
  const int E = 2 * Ar::L;
  for (int part = 0; part < 2; ++part) {
    typename Ar::pacc a, b;
    Ar::pzero(a);
    Ar::pzero(b);
    for (int i = 0; i < n; ++i) Ar::mac_part(kFp, (i < split) ? a : b, load<Ar>(x + i * E), load<Ar>(y + i * E), part);
    Ar::pcombine(kFp, a, b);
    Ar::pfinal(kFp, a, out + part * Ar::L);
  }
}

// out = y - sum_i r_i x_i (complex), through part accumulators
template <class Ar>
void axpy_parts(int n, const double* y, const double* r, const double* x, double* out) {
  const int E = 2 * Ar::L;
  for (int part = 0; part < 2; ++part) {
    typename Ar::pacc a;
    Ar::pzero(a);
    for (int i = 0; i < n; ++i) Ar::mul_acc_part(kFp, a, load<Ar>(r + i * E), load<Ar>(x + i * E), part);
    double yy[4];
    for (int q = 0; q < Ar::L; ++q) yy[q] = y[part * Ar::L + q];
    Ar::psub(kFp, yy, a);
    for (int q = 0; q < Ar::L; ++q) out[part * Ar::L + q] = yy[q];
  }
}

}  // namespace

#define EXPORT extern "C" __attribute__((visibility("default")))

EXPORT int ddqd_host_version() { return 1; }

EXPORT void h_two_sum(double a, double b, double* s, double* e) { mgs::two_sum(kFp, a, b, *s, *e); }
EXPORT void h_two_prod(double a, double b, double* p, double* e) { mgs::two_prod(kFp, a, b, *p, *e); }

// out = sum_i conj(x_i) y_i; elements [0, split) and [split, n) go to two accumulators
// that are then combined (as the kernels combine partial sums).
EXPORT void h_dot(int L, int n, int split, const double* x, const double* y, double* out) {
  if (L == 2)
    dot<mgs::DD>(n, split, x, y, out, false);
  else
    dot<mgs::QD>(n, split, x, y, out, false);
}
EXPORT void h_norm2(int L, int n, int split, const double* x, double* out) {
  if (L == 2)
    dot<mgs::DD>(n, split, x, x, out, true);
  else
    dot<mgs::QD>(n, split, x, x, out, true);
}
// out = y - c x
EXPORT void h_update(int L, const double* y, const double* c, const double* x, double* out) {
  if (L == 2) {
    auto v = load<mgs::DD>(y);
    mgs::DD::update(kFp, v, load<mgs::DD>(c), load<mgs::DD>(x));
    store<mgs::DD>(out, v);
  } else {
    auto v = load<mgs::QD>(y);
    mgs::QD::update(kFp, v, load<mgs::QD>(c), load<mgs::QD>(x));
    store<mgs::QD>(out, v);
  }
}
// out = a / r (a complex, r real)
EXPORT void h_div_real(int L, const double* a, const double* r, double* out) {
  if (L == 2) {
    auto rr = load_real<mgs::DD>(r);
    store<mgs::DD>(out, mgs::DD::div_real(kFp, load<mgs::DD>(a), rr, mgs::DD::inv_lead(rr)));
  } else {
    auto rr = load_real<mgs::QD>(r);
    store<mgs::QD>(out, mgs::QD::div_real(kFp, load<mgs::QD>(a), rr, mgs::QD::inv_lead(rr)));
  }
}
EXPORT void h_mul_real(int L, const double* a, const double* r, double* out) {
  if (L == 2)
    store<mgs::DD>(out, mgs::DD::mul_real(kFp, load<mgs::DD>(a), load_real<mgs::DD>(r)));
  else
    store<mgs::QD>(out, mgs::QD::mul_real(kFp, load<mgs::QD>(a), load_real<mgs::QD>(r)));
}
EXPORT void h_sqrt(int L, const double* s, double* out) {
  if (L == 2)
    store_real<mgs::DD>(out, mgs::DD::sqrt(kFp, load_real<mgs::DD>(s)));
  else
    store_real<mgs::QD>(out, mgs::QD::sqrt(kFp, load_real<mgs::QD>(s)));
}

EXPORT void h_dot_parts(int L, int n, int split, const double* x, const double* y, double* out) {
  if (L == 2)
    dot_parts<mgs::DD>(n, split, x, y, out);
  else
    dot_parts<mgs::QD>(n, split, x, y, out);
}
EXPORT void h_axpy_parts(int L, int n, const double* y, const double* r, const double* x, double* out) {
  if (L == 2)
    axpy_parts<mgs::DD>(n, y, r, x, out);
  else
    axpy_parts<mgs::QD>(n, y, r, x, out);
}
// out = y - c x (QD) as the back substitution's chain forms it: each part is split over
// two accumulators (the seeded one takes the product c_re x_part, the other the cross
// term), merged and renormalised.
EXPORT void h_update_split_qd(const double* y, const double* c, const double* x, double* out) {
  using Q = mgs::QD;
  const auto cc = load<Q>(c), xx = load<Q>(x);
  for (int part = 0; part < 2; ++part) {
    Q::pacc a, b;
    Q::pseed(a, y + part * 4);
    Q::mul_sub_half(kFp, a, cc, xx, part, 0);
    Q::pzero(b);
    Q::mul_sub_half(kFp, b, cc, xx, part, 1);
    Q::pcombine(kFp, a, b);
    Q::pfinal(kFp, a, out + part * 4);
  }
}
