// Double-double (DD) and quad-double (QD) complex arithmetic on FP64 limbs for sm_103a.
//
// Error-free transforms (Knuth's two-sum, Dekker's fast two-sum, the FMA two-product)
// are the only building blocks; every operation is written for this project.
//
// Cost model of this GPU (measured): an FP64 warp-instruction occupies the SM
// sub-partition's FP64 unit for 64 cycles when it is a DFMA and 76 cycles when it is a
// DADD or DMUL, while integer and logic instructions cost about 2 cycles.  Hence:
//   * every FP64 add, subtract and multiply is issued in FMA form through Fp, whose `one`
//     and `nzero` (1.0 and -0.0) are run-time values the compiler cannot fold back;
//   * the magnitude test of a two-sum is an integer comparison of the bit patterns, so
//     two-sum costs 3 FP64 instructions instead of Knuth's branch-free 6;
//   * negation is an operand modifier (free).
//
// Limb layout of a complex element with L limbs per real part (L = 2 DD, L = 4 QD):
//   v[0..L-1] = real part (largest limb first), v[L..2L-1] = imaginary part.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

#if !defined(__CUDACC__)
// Plain C++ build of this header (host tests of the arithmetic): the device qualifiers
// vanish and the intrinsics map to their correctly rounded C++ counterparts, so host
// results are bit-identical to the GPU's.
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace mgs {

#if defined(__CUDA_ARCH__)
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ long long bits_of(double a) { return __double_as_longlong(a); }
__device__ __forceinline__ double rcp_rn(double a) { return __drcp_rn(a); }
__device__ __forceinline__ double sqrt_rn(double a) { return __dsqrt_rn(a); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ unsigned hi_word(double a) { return (unsigned)__double2hiint(a); }
__device__ __forceinline__ double with_hi_word(double a, unsigned hi) {
  return __hiloint2double((int)hi, __double2loint(a));
}
#else
__host__ __device__ inline double fma_rn(double a, double b, double c) { return std::fma(a, b, c); }
__host__ __device__ inline long long bits_of(double a) {
  long long v;
  std::memcpy(&v, &a, sizeof v);
  return v;
}
__host__ __device__ inline double rcp_rn(double a) { return 1.0 / a; }
__host__ __device__ inline double sqrt_rn(double a) { return std::sqrt(a); }
__host__ __device__ inline double div_rn(double a, double b) { return a / b; }
__host__ __device__ inline unsigned hi_word(double a) { return (unsigned)((unsigned long long)bits_of(a) >> 32); }
__host__ __device__ inline double with_hi_word(double a, unsigned hi) {
  unsigned long long b = ((unsigned long long)hi << 32) | ((unsigned long long)bits_of(a) & 0xffffffffULL);
  double r;
  std::memcpy(&r, &b, sizeof r);
  return r;
}
#endif

struct Fp {
  double one;    // 1.0 at run time
  double nzero;  // -0.0 at run time (a*b + (-0) == a*b for every a, b)
  __host__ __device__ __forceinline__ double add(double a, double b) const { return fma_rn(a, one, b); }
  __host__ __device__ __forceinline__ double sub(double a, double b) const { return fma_rn(b, -one, a); }
  __host__ __device__ __forceinline__ double mul(double a, double b) const { return fma_rn(a, b, nzero); }
  __host__ __device__ __forceinline__ double fma(double a, double b, double c) const { return fma_rn(a, b, c); }
};

// Exponent order for fast two-sum: the sign-cleared high words (exponent and the top 20
// mantissa bits) compared as unsigned integers.  If they are equal the exponents are
// equal, which is all Dekker's condition needs.  Done on the high 32-bit words on
// purpose: a 64-bit sign-masked compare is recognised as |a| >= |b| and compiled to
// FP64-pipe instructions (measured: 2 extra per two-sum).
__host__ __device__ __forceinline__ bool mag_ge(double a, double b) {
  return (hi_word(a) & 0x7fffffffu) >= (hi_word(b) & 0x7fffffffu);
}

// s = fl(a + b), e = (a + b) - s exactly.  Orders the operands by magnitude, then runs
// Dekker's fast two-sum (exact when the first operand is the larger one).
__host__ __device__ __forceinline__ void two_sum(const Fp& f, double a, double b, double& s, double& e) {
  const bool keep = mag_ge(a, b);
  const double x = keep ? a : b;
  const double y = keep ? b : a;
  s = f.add(x, y);
  const double t = f.sub(s, x);
  e = f.sub(y, t);
}

// Dekker's fast two-sum; requires |a| >= |b| (or a == 0).
__host__ __device__ __forceinline__ void fast_two_sum(const Fp& f, double a, double b, double& s, double& e) {
  s = f.add(a, b);
  const double t = f.sub(s, a);
  e = f.sub(b, t);
}

// p = fl(a * b), e = a * b - p exactly (barring underflow).
__host__ __device__ __forceinline__ void two_prod(const Fp& f, double a, double b, double& p, double& e) {
  p = f.mul(a, b);
  e = f.fma(a, b, -p);
}

// v or -v, chosen on the integer pipe (an exclusive-or of the sign bit in the high word).
__host__ __device__ __forceinline__ double flip_if(double v, bool neg) {
  return with_hi_word(v, hi_word(v) ^ (neg ? 0x80000000u : 0u));
}

__host__ __device__ __forceinline__ bool finite64(double a) {
  return (hi_word(a) & 0x7ff00000u) != 0x7ff00000u;
}

// =====================================================================================
// Complex double (one limb): the plain FP64 arithmetic of the paper's "complex double"
// runs (Sections 4 and 8), with the same interface as DD and QD.
// =====================================================================================
struct D {
  static constexpr int L = 1;
  static constexpr int ACC = 2;
  struct real {
    double h;
  };
  struct elem {
    double v[2];  // re, im
  };
  struct acc {
    double r, i;
  };
  struct pacc {
    double s;
  };
  static constexpr int PACC = 1;
  // FP64 instructions of mac_part and of pcombine (work-mapping choices weigh with them)
  static constexpr int kMacOps = 2, kCombineOps = 1;
  __host__ __device__ static __forceinline__ void pzero(pacc& a) { a.s = 0.0; }
  // part 0: a += xr yr + xi yi;  part 1: a += xr yi - xi yr
  __host__ __device__ static __forceinline__ void mac_part(const Fp& f, pacc& a, const elem& x, const elem& y,
                                                          int part) {
    const bool im = part != 0;
    a.s = f.fma(x.v[0], im ? y.v[1] : y.v[0], a.s);
    a.s = f.fma(flip_if(x.v[1], im), im ? y.v[0] : y.v[1], a.s);
  }
  // part 0: a += rr xr - ri xi;  part 1: a += rr xi + ri xr
  __host__ __device__ static __forceinline__ void mul_acc_part(const Fp& f, pacc& a, const elem& r, const elem& x,
                                                              int part) {
    const bool im = part != 0;
    a.s = f.fma(r.v[0], im ? x.v[1] : x.v[0], a.s);
    a.s = f.fma(flip_if(r.v[1], !im), im ? x.v[0] : x.v[1], a.s);
  }
  __host__ __device__ static __forceinline__ void pcombine(const Fp& f, pacc& a, const pacc& b) {
    a.s = f.add(a.s, b.s);
  }
  __host__ __device__ static __forceinline__ void pfinal(const Fp&, const pacc& a, double* o) { o[0] = a.s; }
  __host__ __device__ static __forceinline__ void psub(const Fp& f, double* y, const pacc& a) {
    y[0] = f.sub(y[0], a.s);
  }
  __host__ __device__ static __forceinline__ real re(const elem& x) { return real{x.v[0]}; }
  // one part of y := y - c x
  __host__ __device__ static __forceinline__ void update_part(const Fp& f, elem& y, const elem& c, const elem& x,
                                                             int part) {
    const bool im = part != 0;
    double t = im ? y.v[1] : y.v[0];
    t = f.fma(-c.v[0], im ? x.v[1] : x.v[0], t);
    t = f.fma(flip_if(c.v[1], im), im ? x.v[0] : x.v[1], t);
    y.v[0] = im ? y.v[0] : t;
    y.v[1] = im ? t : y.v[1];
  }
  // y := y - c x, both parts (the operations of update_part, in the same order)
  __host__ __device__ static __forceinline__ void update(const Fp& f, elem& y, const elem& c, const elem& x) {
    y.v[0] = f.fma(c.v[1], x.v[1], f.fma(-c.v[0], x.v[0], y.v[0]));
    y.v[1] = f.fma(-c.v[1], x.v[0], f.fma(-c.v[0], x.v[1], y.v[1]));
  }
  __host__ __device__ static __forceinline__ double inv_lead(const real& r) { return rcp_rn(r.h); }
  __host__ __device__ static __forceinline__ void div_real_part(const Fp&, elem& q, const elem& a, const real& r,
                                                               double, int part) {
    const bool im = part != 0;
    const double v = div_rn(im ? a.v[1] : a.v[0], r.h);
    q.v[0] = im ? q.v[0] : v;
    q.v[1] = im ? v : q.v[1];
  }
  __host__ __device__ static __forceinline__ void mul_real_part(const Fp& f, elem& q, const elem& a, const real& r,
                                                               int part) {
    const bool im = part != 0;
    const double v = f.mul(im ? a.v[1] : a.v[0], r.h);
    q.v[0] = im ? q.v[0] : v;
    q.v[1] = im ? v : q.v[1];
  }
  __host__ __device__ static __forceinline__ elem from_real(const real& r) { return elem{{r.h, 0.0}}; }
  __host__ __device__ static __forceinline__ real inv_real(const Fp&, const real& r) { return real{div_rn(1.0, r.h)}; }
  __host__ __device__ static __forceinline__ real sqrt(const Fp&, const real& s) {
    return real{s.h > 0.0 ? sqrt_rn(s.h) : 0.0};
  }
  __host__ __device__ static __forceinline__ bool positive(const real& r) { return r.h > 0.0 && finite64(r.h); }
};

// =====================================================================================
// Double-double
// =====================================================================================
struct DD {
  static constexpr int L = 2;
  static constexpr int ACC = 4;  // doubles in a complex dot-product accumulator

  struct real {
    double h, l;
  };
  struct elem {
    double v[4];  // re_h, re_l, im_h, im_l
  };
  // Compensated (Dot2-style) accumulator: the value is S + C where S collects the
  // leading products through error-free two-sums and C every rounding error and every
  // low-order product; one per real/imaginary part.
  struct acc {
    double sr, cr, si, ci;
  };

  __host__ __device__ static __forceinline__ void zero(acc& a) { a.sr = a.cr = a.si = a.ci = 0.0; }

  // S + C += a * b  with a = (ah, al), b = (bh, bl): 9 FP64 instructions.
  __host__ __device__ static __forceinline__ void term(const Fp& f, double& S, double& C, double ah, double al, double bh,
                                              double bl) {
    double p, e, s, t;
    two_prod(f, ah, bh, p, e);
    two_sum(f, S, p, s, t);
    S = s;
    C = f.fma(ah, bl, C);
    C = f.fma(al, bh, C);
    C = f.add(C, e);
    C = f.add(C, t);
  }

  // One part (real or imaginary) of a dot-product accumulator: S + C.
  struct pacc {
    double S, C;
  };
  static constexpr int PACC = 2;
  static constexpr int kMacOps = 18, kCombineOps = 5;  // mac_part, pcombine
  __host__ __device__ static __forceinline__ void pzero(pacc& a) { a.S = a.C = 0.0; }
  // part 0: a += Re(conj(x) y) = xr yr + xi yi;  part 1: a += Im(conj(x) y) = xr yi - xi yr
  __host__ __device__ static __forceinline__ void mac_part(const Fp& f, pacc& a, const elem& x, const elem& y,
                                                          int part) {
    const bool im = part != 0;
    const double y1h = im ? y.v[2] : y.v[0], y1l = im ? y.v[3] : y.v[1];
    const double y2h = im ? y.v[0] : y.v[2], y2l = im ? y.v[1] : y.v[3];
    const double x2h = flip_if(x.v[2], im), x2l = flip_if(x.v[3], im);
    term(f, a.S, a.C, x.v[0], x.v[1], y1h, y1l);
    term(f, a.S, a.C, x2h, x2l, y2h, y2l);
  }
  // part 0: a += Re(r x) = rr xr - ri xi;  part 1: a += Im(r x) = rr xi + ri xr
  __host__ __device__ static __forceinline__ void mul_acc_part(const Fp& f, pacc& a, const elem& r, const elem& x,
                                                              int part) {
    const bool im = part != 0;
    const double x1h = im ? x.v[2] : x.v[0], x1l = im ? x.v[3] : x.v[1];
    const double x2h = im ? x.v[0] : x.v[2], x2l = im ? x.v[1] : x.v[3];
    const double r2h = flip_if(r.v[2], !im), r2l = flip_if(r.v[3], !im);
    term(f, a.S, a.C, r.v[0], r.v[1], x1h, x1l);
    term(f, a.S, a.C, r2h, r2l, x2h, x2l);
  }
  __host__ __device__ static __forceinline__ void pcombine(const Fp& f, pacc& a, const pacc& b) {
    double s, t;
    two_sum(f, a.S, b.S, s, t);
    a.S = s;
    a.C = f.add(f.add(a.C, b.C), t);
  }
  __host__ __device__ static __forceinline__ void pfinal(const Fp& f, const pacc& a, double* o) {
    two_sum(f, a.S, a.C, o[0], o[1]);
  }
  // y := y - a for one part (y: L limbs)
  __host__ __device__ static __forceinline__ void psub(const Fp& f, double* y, const pacc& a) {
    double s, t;
    two_sum(f, y[0], -a.S, s, t);
    double lo = f.sub(y[1], a.C);
    lo = f.add(lo, t);
    two_sum(f, s, lo, y[0], y[1]);
  }

  // acc += conj(x) * y   (x^H y convention)
  __host__ __device__ static __forceinline__ void mac_conj(const Fp& f, acc& a, const elem& x, const elem& y) {
    term(f, a.sr, a.cr, x.v[0], x.v[1], y.v[0], y.v[1]);
    term(f, a.sr, a.cr, x.v[2], x.v[3], y.v[2], y.v[3]);
    term(f, a.si, a.ci, x.v[0], x.v[1], y.v[2], y.v[3]);
    term(f, a.si, a.ci, -x.v[2], -x.v[3], y.v[0], y.v[1]);
  }

  // acc.re += |x|^2
  __host__ __device__ static __forceinline__ void mac_norm(const Fp& f, acc& a, const elem& x) {
    term(f, a.sr, a.cr, x.v[0], x.v[1], x.v[0], x.v[1]);
    term(f, a.sr, a.cr, x.v[2], x.v[3], x.v[2], x.v[3]);
  }

  __host__ __device__ static __forceinline__ void combine(const Fp& f, acc& a, const acc& b) {
    double s, t;
    two_sum(f, a.sr, b.sr, s, t);
    a.sr = s;
    a.cr = f.add(f.add(a.cr, b.cr), t);
    two_sum(f, a.si, b.si, s, t);
    a.si = s;
    a.ci = f.add(f.add(a.ci, b.ci), t);
  }

  __host__ __device__ static __forceinline__ elem finalize(const Fp& f, const acc& a) {
    elem r;
    two_sum(f, a.sr, a.cr, r.v[0], r.v[1]);
    two_sum(f, a.si, a.ci, r.v[2], r.v[3]);
    return r;
  }

  __host__ __device__ static __forceinline__ real re(const elem& x) { return real{x.v[0], x.v[1]}; }

  // y := y - c * x  (complex), per part: y - (c.re x.re - c.im x.im) etc.; 42 FP64 ops.
  __host__ __device__ static __forceinline__ void upd_part(const Fp& f, double& yh, double& yl, double c1h, double c1l,
                                                  double x1h, double x1l, double c2h, double c2l, double x2h,
                                                  double x2l) {
    // y - c1*x1 + c2*x2
    double p1, e1, p2, e2, s, t1, t2;
    two_prod(f, c1h, x1h, p1, e1);
    two_prod(f, c2h, x2h, p2, e2);
    two_sum(f, yh, -p1, s, t1);
    two_sum(f, s, p2, s, t2);
    double lo = f.fma(-c1h, x1l, yl);
    lo = f.fma(-c1l, x1h, lo);
    lo = f.fma(c2h, x2l, lo);
    lo = f.fma(c2l, x2h, lo);
    lo = f.sub(lo, e1);
    lo = f.add(lo, e2);
    lo = f.add(lo, t1);
    lo = f.add(lo, t2);
    two_sum(f, s, lo, yh, yl);
  }
  __host__ __device__ static __forceinline__ void update(const Fp& f, elem& y, const elem& c, const elem& x) {
    // re: y.re - c.re x.re + c.im x.im ; im: y.im - c.re x.im - c.im x.re
    upd_part(f, y.v[0], y.v[1], c.v[0], c.v[1], x.v[0], x.v[1], c.v[2], c.v[3], x.v[2], x.v[3]);
    upd_part(f, y.v[2], y.v[3], c.v[0], c.v[1], x.v[2], x.v[3], -c.v[2], -c.v[3], x.v[0], x.v[1]);
  }

  // One part (0 real, 1 imaginary) of y := y - c x.  Operands are picked with selects
  // and sign flips on the integer pipe, so lanes working on different parts execute the
  // same instructions.
  __host__ __device__ static __forceinline__ void update_part(const Fp& f, elem& y, const elem& c, const elem& x,
                                                             int part) {
    const bool im = part != 0;
    double yh = im ? y.v[2] : y.v[0], yl = im ? y.v[3] : y.v[1];
    const double x1h = im ? x.v[2] : x.v[0], x1l = im ? x.v[3] : x.v[1];
    const double x2h = im ? x.v[0] : x.v[2], x2l = im ? x.v[1] : x.v[3];
    const double c2h = flip_if(c.v[2], im), c2l = flip_if(c.v[3], im);
    upd_part(f, yh, yl, c.v[0], c.v[1], x1h, x1l, c2h, c2l, x2h, x2l);
    y.v[0] = im ? y.v[0] : yh;
    y.v[1] = im ? y.v[1] : yl;
    y.v[2] = im ? yh : y.v[2];
    y.v[3] = im ? yl : y.v[3];
  }

  // a / r for real a, r with inv ~ 1/r.h: quotient digit, exact remainder, second digit.
  __host__ __device__ static __forceinline__ void div_part(const Fp& f, double ah, double al, const real& r, double inv,
                                                  double& qh, double& ql) {
    const double q1 = f.mul(ah, inv);
    double p, e;
    two_prod(f, q1, r.h, p, e);
    double t = f.sub(ah, p);
    t = f.sub(t, e);
    t = f.add(t, al);
    t = f.fma(-q1, r.l, t);
    const double q2 = f.mul(t, inv);
    fast_two_sum(f, q1, q2, qh, ql);
  }
  __host__ __device__ static __forceinline__ double inv_lead(const real& r) { return rcp_rn(r.h); }
  __host__ __device__ static __forceinline__ elem div_real(const Fp& f, const elem& a, const real& r, double inv) {
    elem q;
    div_part(f, a.v[0], a.v[1], r, inv, q.v[0], q.v[1]);
    div_part(f, a.v[2], a.v[3], r, inv, q.v[2], q.v[3]);
    return q;
  }

  // One part of a / r (r real) written into q.
  __host__ __device__ static __forceinline__ void div_real_part(const Fp& f, elem& q, const elem& a, const real& r,
                                                               double inv, int part) {
    const bool im = part != 0;
    double qh, ql;
    div_part(f, im ? a.v[2] : a.v[0], im ? a.v[3] : a.v[1], r, inv, qh, ql);
    q.v[0] = im ? q.v[0] : qh;
    q.v[1] = im ? q.v[1] : ql;
    q.v[2] = im ? qh : q.v[2];
    q.v[3] = im ? ql : q.v[3];
  }

  // DD product of two reals.
  __host__ __device__ static __forceinline__ void mul_part(const Fp& f, double ah, double al, const real& b, double& rh,
                                                  double& rl) {
    double p, e;
    two_prod(f, ah, b.h, p, e);
    e = f.fma(ah, b.l, e);
    e = f.fma(al, b.h, e);
    fast_two_sum(f, p, e, rh, rl);
  }
  __host__ __device__ static __forceinline__ elem mul_real(const Fp& f, const elem& a, const real& r) {
    elem q;
    mul_part(f, a.v[0], a.v[1], r, q.v[0], q.v[1]);
    mul_part(f, a.v[2], a.v[3], r, q.v[2], q.v[3]);
    return q;
  }
  __host__ __device__ static __forceinline__ void mul_real_part(const Fp& f, elem& q, const elem& a, const real& r,
                                                               int part) {
    const bool im = part != 0;
    double qh, ql;
    mul_part(f, im ? a.v[2] : a.v[0], im ? a.v[3] : a.v[1], r, qh, ql);
    q.v[0] = im ? q.v[0] : qh;
    q.v[1] = im ? q.v[1] : ql;
    q.v[2] = im ? qh : q.v[2];
    q.v[3] = im ? ql : q.v[3];
  }
  // real part as a real, real-valued element
  __host__ __device__ static __forceinline__ elem from_real(const real& r) { return elem{{r.h, r.l, 0.0, 0.0}}; }
  __host__ __device__ static __forceinline__ real inv_real(const Fp& f, const real& r) {
    const double inv = inv_lead(r);
    double qh, ql;
    div_part(f, 1.0, 0.0, r, inv, qh, ql);
    return real{qh, ql};
  }

  // Square root of s >= 0: one Newton step x + (s - x^2) / (2x) on the rounded double root.
  __host__ __device__ static __forceinline__ real sqrt(const Fp& f, const real& s) {
    if (!(s.h > 0.0)) return real{0.0, 0.0};
    const double x = sqrt_rn(s.h);
    double p, e;
    two_prod(f, x, x, p, e);
    double d = f.sub(s.h, p);
    d = f.sub(d, e);
    d = f.add(d, s.l);
    const double c = div_rn(d, f.add(x, x));
    real r;
    fast_two_sum(f, x, c, r.h, r.l);
    return r;
  }

  __host__ __device__ static __forceinline__ bool positive(const real& r) { return r.h > 0.0 && finite64(r.h); }
};

// =====================================================================================
// Quad-double
// =====================================================================================
struct QD {
  static constexpr int L = 4;
  static constexpr int ACC = 8;

  struct real {
    double x[4];
  };
  struct elem {
    double v[8];  // re0..re3, im0..im3
  };
  // Cascaded accumulator (K-fold compensated summation with K = 4): level 0 collects the
  // leading terms through two-sums, the error of every two-sum at level i goes to level
  // i+1, level 3 is a plain sum.  Value = s0 + s1 + s2 + s3.
  struct part_t {
    double s[4];
  };
  struct acc {
    part_t r, i;
  };

  template <int LV>
  __host__ __device__ static __forceinline__ void put(const Fp& f, part_t& a, double v) {
    if constexpr (LV < 3) {
      double s, t;
      two_sum(f, a.s[LV], v, s, t);
      a.s[LV] = s;
      put<LV + 1>(f, a, t);
    } else {
      a.s[3] = f.add(a.s[3], v);
    }
  }

  template <int LV>
  __host__ __device__ static __forceinline__ void put_prod(const Fp& f, part_t& a, double x, double y) {
    double p, e;
    two_prod(f, x, y, p, e);
    put<LV>(f, a, p);
    put<LV + 1>(f, a, e);
  }

  // a += x * y for QD reals x, y (terms of order 0..3; order >= 4 is below QD precision).
  __host__ __device__ static __forceinline__ void prod(const Fp& f, part_t& a, const double* x, const double* y) {
    put_prod<0>(f, a, x[0], y[0]);
    put_prod<1>(f, a, x[0], y[1]);
    put_prod<1>(f, a, x[1], y[0]);
    put_prod<2>(f, a, x[0], y[2]);
    put_prod<2>(f, a, x[1], y[1]);
    put_prod<2>(f, a, x[2], y[0]);
    a.s[3] = f.fma(x[0], y[3], a.s[3]);
    a.s[3] = f.fma(x[1], y[2], a.s[3]);
    a.s[3] = f.fma(x[2], y[1], a.s[3]);
    a.s[3] = f.fma(x[3], y[0], a.s[3]);
  }
  __host__ __device__ static __forceinline__ void prod_neg(const Fp& f, part_t& a, const double* x, const double* y) {
    const double nx[4] = {-x[0], -x[1], -x[2], -x[3]};
    prod(f, a, nx, y);
  }

  __host__ __device__ static __forceinline__ void zero(acc& a) {
#pragma unroll
    for (int i = 0; i < 4; ++i) a.r.s[i] = a.i.s[i] = 0.0;
  }

  using pacc = part_t;
  static constexpr int PACC = 4;
  static constexpr int kMacOps = 140, kCombineOps = 22;  // mac_part, pcombine
  __host__ __device__ static __forceinline__ void pzero(pacc& a) {
#pragma unroll
    for (int i = 0; i < 4; ++i) a.s[i] = 0.0;
  }
  // part 0: a += xr yr + xi yi;  part 1: a += xr yi - xi yr
  __host__ __device__ static __forceinline__ void mac_part(const Fp& f, pacc& a, const elem& x, const elem& y,
                                                          int part) {
    const bool im = part != 0;
    double y1[4], y2[4], x2[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      y1[i] = im ? y.v[4 + i] : y.v[i];
      y2[i] = im ? y.v[i] : y.v[4 + i];
      x2[i] = flip_if(x.v[4 + i], im);
    }
    prod(f, a, x.v, y1);
    prod(f, a, x2, y2);
  }
  // part 0: a += rr xr - ri xi;  part 1: a += rr xi + ri xr
  __host__ __device__ static __forceinline__ void mul_acc_part(const Fp& f, pacc& a, const elem& r, const elem& x,
                                                              int part) {
    const bool im = part != 0;
    double x1[4], x2[4], r2[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      x1[i] = im ? x.v[4 + i] : x.v[i];
      x2[i] = im ? x.v[i] : x.v[4 + i];
      r2[i] = flip_if(r.v[4 + i], !im);
    }
    prod(f, a, r.v, x1);
    prod(f, a, r2, x2);
  }
  // One half of part `part` of a -= r x: half 0 subtracts the product rr x_part, half 1
  // the cross term (ri xi for the real part, ri xr for the imaginary part); the two halves
  // run on two lanes and are merged, which halves a dependent update chain.
  __host__ __device__ static __forceinline__ void mul_sub_half(const Fp& f, pacc& a, const elem& r, const elem& x,
                                                              int part, int half) {
    const bool im = part != 0, h1 = half != 0;
    double u[4], v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      u[i] = h1 ? flip_if(r.v[4 + i], im) : -r.v[i];
      v[i] = (im != h1) ? x.v[4 + i] : x.v[i];
    }
    prod(f, a, u, v);
  }
  // An accumulator holding the normalised value y (L limbs).
  __host__ __device__ static __forceinline__ void pseed(pacc& a, const double* y) {
#pragma unroll
    for (int i = 0; i < 4; ++i) a.s[i] = y[i];
  }
  __host__ __device__ static __forceinline__ void pcombine(const Fp& f, pacc& a, const pacc& b) { merge(f, a, b); }
  __host__ __device__ static __forceinline__ void pfinal(const Fp& f, const pacc& a, double* o) { renorm(f, a, o); }
  __host__ __device__ static __forceinline__ void psub(const Fp& f, double* y, const pacc& a) {
    part_t t{{y[0], y[1], y[2], y[3]}};
    put<0>(f, t, -a.s[0]);
    put<1>(f, t, -a.s[1]);
    put<2>(f, t, -a.s[2]);
    put<3>(f, t, -a.s[3]);
    renorm(f, t, y);
  }

  __host__ __device__ static __forceinline__ void mac_conj(const Fp& f, acc& a, const elem& x, const elem& y) {
    prod(f, a.r, x.v, y.v);          // xr yr
    prod(f, a.r, x.v + 4, y.v + 4);  // xi yi
    prod(f, a.i, x.v, y.v + 4);      // xr yi
    prod_neg(f, a.i, x.v + 4, y.v);  // -xi yr
  }

  __host__ __device__ static __forceinline__ void mac_norm(const Fp& f, acc& a, const elem& x) {
    prod(f, a.r, x.v, x.v);
    prod(f, a.r, x.v + 4, x.v + 4);
  }

  __host__ __device__ static __forceinline__ void merge(const Fp& f, part_t& a, const part_t& b) {
    put<0>(f, a, b.s[0]);
    put<1>(f, a, b.s[1]);
    put<2>(f, a, b.s[2]);
    put<3>(f, a, b.s[3]);
  }
  __host__ __device__ static __forceinline__ void combine(const Fp& f, acc& a, const acc& b) {
    merge(f, a.r, b.r);
    merge(f, a.i, b.i);
  }

  // Accumulator levels -> normalised 4-limb expansion (two two-sum sweeps).
  __host__ __device__ static __forceinline__ void renorm(const Fp& f, const part_t& a, double* o) {
    double s0, s1, s2, s3;
    two_sum(f, a.s[2], a.s[3], s2, s3);
    two_sum(f, a.s[1], s2, s1, s2);
    two_sum(f, a.s[0], s1, s0, s1);
    two_sum(f, s1, s2, s1, s2);
    two_sum(f, s2, s3, s2, s3);
    two_sum(f, s0, s1, s0, s1);
    two_sum(f, s1, s2, s1, s2);
    o[0] = s0;
    o[1] = s1;
    o[2] = s2;
    o[3] = s3;
  }

  __host__ __device__ static __forceinline__ elem finalize(const Fp& f, const acc& a) {
    elem r;
    renorm(f, a.r, r.v);
    renorm(f, a.i, r.v + 4);
    return r;
  }

  __host__ __device__ static __forceinline__ real re(const elem& x) { return real{{x.v[0], x.v[1], x.v[2], x.v[3]}}; }

  // y := y - c x
  __host__ __device__ static __forceinline__ void update(const Fp& f, elem& y, const elem& c, const elem& x) {
    part_t pr{{y.v[0], y.v[1], y.v[2], y.v[3]}};
    part_t pi{{y.v[4], y.v[5], y.v[6], y.v[7]}};
    prod_neg(f, pr, c.v, x.v);          // - cr xr
    prod(f, pr, c.v + 4, x.v + 4);      // + ci xi
    prod_neg(f, pi, c.v, x.v + 4);      // - cr xi
    prod_neg(f, pi, c.v + 4, x.v);      // - ci xr
    renorm(f, pr, y.v);
    renorm(f, pi, y.v + 4);
  }

  // One part (0 real, 1 imaginary) of y := y - c x (see DD::update_part).
  __host__ __device__ static __forceinline__ void update_part(const Fp& f, elem& y, const elem& c, const elem& x,
                                                             int part) {
    const bool im = part != 0;
    part_t s;
    double x1[4], x2[4], c2[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      s.s[i] = im ? y.v[4 + i] : y.v[i];
      x1[i] = im ? x.v[4 + i] : x.v[i];
      x2[i] = im ? x.v[i] : x.v[4 + i];
      c2[i] = flip_if(c.v[4 + i], im);
    }
    prod_neg(f, s, c.v, x1);
    prod(f, s, c2, x2);
    double o[4];
    renorm(f, s, o);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      y.v[i] = im ? y.v[i] : o[i];
      y.v[4 + i] = im ? o[i] : y.v[4 + i];
    }
  }

  __host__ __device__ static __forceinline__ double inv_lead(const real& r) { return rcp_rn(r.x[0]); }

  // a / r: long division with an exactly tracked remainder.  inv ~ 1/r.x[0] is refined
  // to a double-double reciprocal (one Newton correction), which yields two 104-bit
  // double-double quotient digits; a last 53-bit digit takes the error below 2^-210.
  __host__ __device__ static __forceinline__ void div_part(const Fp& f, const double* a, const real& r, double inv,
                                                           double* q) {
    double e = f.fma(-r.x[0], inv, f.one);  // 1 - r inv, exact enough: |e| ~ 2^-53
    e = f.fma(-r.x[1], inv, e);
    const double ilo = f.mul(inv, e);  // (inv, ilo) ~ 1/r to 2^-104
    part_t rem{{a[0], a[1], a[2], a[3]}};
    double d[4];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      // double-double digit: leading two limbs of the (normalised) remainder times (inv, ilo)
      double p, pe, qh, ql;
      two_prod(f, rem.s[0], inv, p, pe);
      pe = f.fma(rem.s[0], ilo, pe);
      pe = f.fma(rem.s[1], inv, pe);
      fast_two_sum(f, p, pe, qh, ql);
      d[2 * t] = qh;
      d[2 * t + 1] = ql;
      // rem -= (qh + ql) r, terms of order 0..3
      put_prod<0>(f, rem, -qh, r.x[0]);
      put_prod<1>(f, rem, -qh, r.x[1]);
      put_prod<1>(f, rem, -ql, r.x[0]);
      put_prod<2>(f, rem, -qh, r.x[2]);
      put_prod<2>(f, rem, -ql, r.x[1]);
      rem.s[3] = f.fma(-qh, r.x[3], rem.s[3]);
      rem.s[3] = f.fma(-ql, r.x[2], rem.s[3]);
      renorm(f, rem, rem.s);  // the leading levels cancel; renormalise for the next digit
    }
    // digits sit at levels 0..3; the last single digit is below level 3
    part_t sq{{d[0], d[1], d[2], d[3]}};
    sq.s[3] = f.add(sq.s[3], f.mul(rem.s[0], inv));
    renorm(f, sq, q);
  }
  __host__ __device__ static __forceinline__ elem div_real(const Fp& f, const elem& a, const real& r, double inv) {
    elem q;
    div_part(f, a.v, r, inv, q.v);
    div_part(f, a.v + 4, r, inv, q.v + 4);
    return q;
  }

  __host__ __device__ static __forceinline__ void div_real_part(const Fp& f, elem& q, const elem& a, const real& r,
                                                               double inv, int part) {
    const bool im = part != 0;
    double ai[4], o[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) ai[i] = im ? a.v[4 + i] : a.v[i];
    div_part(f, ai, r, inv, o);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      q.v[i] = im ? q.v[i] : o[i];
      q.v[4 + i] = im ? o[i] : q.v[4 + i];
    }
  }

  __host__ __device__ static __forceinline__ void mulr(const Fp& f, const double* a, const real& b, double* o) {
    part_t p{{0.0, 0.0, 0.0, 0.0}};
    prod(f, p, a, b.x);
    renorm(f, p, o);
  }
  __host__ __device__ static __forceinline__ elem mul_real(const Fp& f, const elem& a, const real& r) {
    elem q;
    mulr(f, a.v, r, q.v);
    mulr(f, a.v + 4, r, q.v + 4);
    return q;
  }

  __host__ __device__ static __forceinline__ void mul_real_part(const Fp& f, elem& q, const elem& a, const real& r,
                                                               int part) {
    const bool im = part != 0;
    double ai[4], o[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) ai[i] = im ? a.v[4 + i] : a.v[i];
    mulr(f, ai, r, o);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      q.v[i] = im ? q.v[i] : o[i];
      q.v[4 + i] = im ? o[i] : q.v[4 + i];
    }
  }
  __host__ __device__ static __forceinline__ elem from_real(const real& r) {
    return elem{{r.x[0], r.x[1], r.x[2], r.x[3], 0.0, 0.0, 0.0, 0.0}};
  }
  __host__ __device__ static __forceinline__ real inv_real(const Fp& f, const real& r) {
    const double one[4] = {1.0, 0.0, 0.0, 0.0};
    real q;
    div_part(f, one, r, inv_lead(r), q.x);
    return q;
  }

  // Square root: Newton x <- x + (s - x^2) / (2x), three steps from the double root
  // (quadratic convergence: 2^-53 -> 2^-106 -> 2^-212, the third absorbs rounding).
  __host__ __device__ static __forceinline__ real sqrt(const Fp& f, const real& s) {
    if (!(s.x[0] > 0.0)) return real{{0.0, 0.0, 0.0, 0.0}};
    real x{{sqrt_rn(s.x[0]), 0.0, 0.0, 0.0}};
#pragma unroll 1
    for (int it = 0; it < 3; ++it) {
      part_t r{{s.x[0], s.x[1], s.x[2], s.x[3]}};
      const double nx[4] = {-x.x[0], -x.x[1], -x.x[2], -x.x[3]};
      prod(f, r, nx, x.x);  // s - x^2
      double rr[4];
      renorm(f, r, rr);
      real twox{{f.add(x.x[0], x.x[0]), f.add(x.x[1], x.x[1]), f.add(x.x[2], x.x[2]), f.add(x.x[3], x.x[3])}};
      double c[4];
      div_part(f, rr, twox, rcp_rn(twox.x[0]), c);
      part_t sum{{x.x[0], x.x[1], x.x[2], x.x[3]}};
      put<0>(f, sum, c[0]);
      put<1>(f, sum, c[1]);
      put<2>(f, sum, c[2]);
      put<3>(f, sum, c[3]);
      renorm(f, sum, x.x);
    }
    return x;
  }

  __host__ __device__ static __forceinline__ bool positive(const real& r) { return r.x[0] > 0.0 && finite64(r.x[0]); }
};

}  // namespace mgs
