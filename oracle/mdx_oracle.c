/*
 * Oracle for complex double-double (DD) / quad-double (QD) modified Gram-Schmidt
 * least squares: the plain, slow, sequential CPU definition that the CUDA path is
 * checked against.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or load this
 * file; only the tests, the smoke check and the CPU-baseline leg of the benchmark do.
 * It shares no code, header or constant with the CUDA library.
 *
 * What it computes (Verschelde & Yoffe, "Orthogonalization on a GPGPU with double
 * double and quad double arithmetic"):
 *   - Section 3, Figure 1: modified Gram-Schmidt, for k = 1..n:
 *         r_kk = sqrt(a_k^H a_k);  q_k = a_k / r_kk;
 *         for j > k:  r_kj = q_k^H a_j;  a_j = a_j - r_kj q_k
 *     with x^H y = sum_l conj(x_l) y_l (Section 3, inner-product convention).
 *   - Section 3, Eq. (1): MGS on the augmented matrix [A b] = [Q q_{n+1}] [[R y],[0 z]],
 *     so that y = Q^H b and ||b - A x||^2 = ||R x - y||^2 + z^2.  The last column is
 *     reduced but not normalised: what remains of it is the residual b - A x, and its
 *     norm is z.
 *   - Section 6, Figure 3: column-oriented back substitution, for k = n..1:
 *         x_k = y_k / r_kk;  for j < k:  y_j = y_j - r_jk x_k.
 *   - Section 4, Eq. (2): the accuracy measure e = max_ij |a_ij - sum_l q_il r_lj|.
 *
 * Arithmetic.  A real number carries L limbs (L = 1 double, 2 double-double,
 * 4 quad-double; L = 8 is also accepted, as a reference of twice quad-double precision
 * for judging a quad-double solve); its value is the exact sum of the limbs.  Every elementary operation
 * (+, -, *) is first evaluated EXACTLY as a floating-point expansion (Shewchuk 1997,
 * "Adaptive precision floating-point arithmetic": error-free two-sum of Knuth, two-product
 * through a fused multiply-add as in Dekker 1971, expansion growth with zero elimination),
 * then rounded to L limbs by peeling off the double nearest to what remains, L times.
 * The result of every operation is therefore the exact result to within about 2^(-53 L)
 * relative.  Division is schoolbook long division with exact remainders (L+1 quotient
 * digits); the square root is Newton's iteration x <- x + (s - x^2)/(2x) from the double
 * square root of the leading limb, with ceil(log2 L)+1 steps.
 *
 * Complex numbers are (re, im) pairs of such reals and use the textbook formulas on top
 * of the rounded real operations.  Sums (norms, inner products) run sequentially over
 * l = 1..m; nothing is blocked, fused or reordered.
 *
 * Memory layout shared with the callers: a complex element is 2L consecutive doubles
 * {re_0..re_{L-1}, im_0..im_{L-1}}; matrices are column-major by element, element (i,j)
 * at base + (j*ld + i)*2L.
 *
 * Build with -O2 -ffp-contract=off (no -ffast-math): the error-free transforms below are
 * only exact when the compiler does not fuse a*b+c behind our back.  oracle_selfcheck()
 * detects a build that does.
 *
 * Planted-mistake builds (-DORACLE_PLANT=k) exist only so the test suite can show that
 * its pins catch a wrong oracle; the default build defines no plant.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORACLE_PLANT
#define ORACLE_PLANT 0
#endif

#define LMAX 8 /* L = 8 (octo-double) serves only as a higher-precision reference */
#define XCAP 1024 /* capacity of an expansion; long sums compress before reaching it */

typedef struct {
  int n;
  double c[XCAP];
} xp; /* nonoverlapping expansion, increasing magnitude, no zero components */

typedef struct {
  double v[LMAX];
} mp; /* L-limb real */

typedef struct {
  mp re, im;
} cx; /* complex */

static int g_overflow = 0; /* set if an expansion ever ran out of room */

/* ---------------------------------------------------------------- error-free transforms */

/* Knuth's two-sum: s = fl(a+b), e = (a+b) - s exactly, for any a, b. */
static void two_sum(double a, double b, double *s, double *e) {
  double x = a + b;
  double bv = x - a;
  double av = x - bv;
  double br = b - bv;
  double ar = a - av;
  *s = x;
  *e = ar + br;
}

/* Two-product through FMA: p = fl(a*b), e = a*b - p exactly (barring underflow). */
static void two_prod(double a, double b, double *p, double *e) {
  double x = a * b;
  *p = x;
#if ORACLE_PLANT == 1
  *e = 0.0; /* planted: drop the rounding error of the product */
#else
  *e = fma(a, b, -x);
#endif
}

/* ---------------------------------------------------------------- expansions */

static void xp_compress(xp *E);

/* E := E + b exactly (Shewchuk's GROW-EXPANSION with zero elimination). */
static void xp_grow(xp *E, double b) {
  if (E->n + 1 > XCAP) {
    xp_compress(E);
    if (E->n + 1 > XCAP) {
      g_overflow = 1;
      return;
    }
  }
  double q = b;
  int k = 0;
  for (int i = 0; i < E->n; ++i) {
    double s, h;
    two_sum(q, E->c[i], &s, &h);
    q = s;
    if (h != 0.0) E->c[k++] = h;
  }
  if (q != 0.0) E->c[k++] = q;
  E->n = k;
}

/* Shewchuk's COMPRESS: same value, fewer components (largest one approximates the sum). */
static void xp_compress(xp *E) {
  int m = E->n;
  if (m < 2) return;
  static __thread double g[XCAP];
  double Q = E->c[m - 1];
  int bottom = m - 1;
  for (int i = m - 2; i >= 0; --i) {
    double s, q;
    two_sum(Q, E->c[i], &s, &q);
    if (q != 0.0) {
      g[bottom--] = s;
      Q = q;
    } else {
      Q = s;
    }
  }
  g[bottom] = Q;
  int top = 0;
  for (int i = bottom + 1; i < m; ++i) {
    double s, q;
    two_sum(g[i], Q, &s, &q);
    if (q != 0.0) E->c[top++] = q;
    Q = s;
  }
  if (Q != 0.0 || top == 0) E->c[top++] = Q;
  if (top == 1 && E->c[0] == 0.0) top = 0;
  E->n = top;
}

/* Approximate value: sum from the smallest component up. */
static double xp_approx(const xp *E) {
  double s = 0.0;
  for (int i = 0; i < E->n; ++i) s += E->c[i];
  return s;
}

static double ulp_of(double x) {
  double a = fabs(x);
  return nextafter(a, INFINITY) - a;
}

/* Round an exact expansion to L limbs: limb i is the double nearest to what the limbs
   before it left over. */
static mp xp_round(const xp *E, int L) {
  static __thread xp R, T;
  mp out;
  memset(&out, 0, sizeof out);
  R.n = E->n;
  memcpy(R.c, E->c, sizeof(double) * (size_t)E->n);
#if ORACLE_PLANT == 7
  int keep = L > 1 ? L - 1 : 1; /* planted: the last limb is never filled */
#else
  int keep = L;
#endif
  for (int i = 0; i < keep; ++i) {
    double x = xp_approx(&R);
    for (int it = 0;; ++it) {
      T.n = R.n;
      memcpy(T.c, R.c, sizeof(double) * (size_t)R.n);
      xp_grow(&T, -x);
      double d = xp_approx(&T);
      if (x == 0.0 || fabs(d) <= 0.5 * ulp_of(x) || it == 4) break;
      x = x + d;
    }
    out.v[i] = x;
    R.n = T.n;
    memcpy(R.c, T.c, sizeof(double) * (size_t)T.n);
  }
  return out;
}

static void xp_add_mp(xp *E, const mp *a, int L, double sign) {
  for (int i = 0; i < L; ++i) xp_grow(E, sign * a->v[i]);
}

/* E += sign * a*b exactly */
static void xp_add_prod(xp *E, const mp *a, const mp *b, int L, double sign) {
  for (int i = 0; i < L; ++i)
    for (int j = 0; j < L; ++j) {
      double p, e;
      two_prod(a->v[i], b->v[j], &p, &e);
      xp_grow(E, sign * p);
      xp_grow(E, sign * e);
    }
}

/* ---------------------------------------------------------------- L-limb reals */

static mp mp_zero(void) {
  mp z;
  memset(&z, 0, sizeof z);
  return z;
}

static mp mp_from_double(double d) {
  mp z = mp_zero();
  z.v[0] = d;
  return z;
}

static double mp_approx(const mp *a, int L) {
  double s = 0.0;
  for (int i = L - 1; i >= 0; --i) s += a->v[i];
  return s;
}

static int mp_finite(const mp *a, int L) {
  for (int i = 0; i < L; ++i)
    if (!isfinite(a->v[i])) return 0;
  return 1;
}

static mp mp_neg(mp a, int L) {
  for (int i = 0; i < L; ++i) a.v[i] = -a.v[i];
  return a;
}

static mp mp_add(mp a, mp b, int L) {
  static __thread xp E;
  E.n = 0;
  xp_add_mp(&E, &a, L, 1.0);
  xp_add_mp(&E, &b, L, 1.0);
  return xp_round(&E, L);
}

static mp mp_sub(mp a, mp b, int L) { return mp_add(a, mp_neg(b, L), L); }

static mp mp_mul(mp a, mp b, int L) {
  static __thread xp E;
  E.n = 0;
  xp_add_prod(&E, &a, &b, L, 1.0);
  return xp_round(&E, L);
}

/* Schoolbook long division: each quotient digit is the leading part of the exact
   remainder divided by the leading limb of b; the remainder is updated exactly. */
static mp mp_div(mp a, mp b, int L) {
  static __thread xp Rm, Qd;
  Rm.n = 0;
  Qd.n = 0;
  xp_add_mp(&Rm, &a, L, 1.0);
#if ORACLE_PLANT == 5
  int digits = 1; /* planted: a single quotient digit */
#else
  int digits = L + 1;
#endif
  for (int d = 0; d < digits; ++d) {
    double qd = xp_approx(&Rm) / b.v[0];
    if (qd == 0.0 || !isfinite(qd)) {
      if (!isfinite(qd)) xp_grow(&Qd, qd);
      break;
    }
    xp_grow(&Qd, qd);
    for (int j = 0; j < L; ++j) {
      double p, e;
      two_prod(qd, b.v[j], &p, &e);
      xp_grow(&Rm, -p);
      xp_grow(&Rm, -e);
    }
  }
  return xp_round(&Qd, L);
}

static mp mp_half(mp a, int L) {
  for (int i = 0; i < L; ++i) a.v[i] *= 0.5; /* exact: power-of-two scaling */
  return a;
}

/* Square root of s >= 0 by Newton's iteration x <- x + (s - x*x) / (2x). */
static mp mp_sqrt(mp s, int L) {
  if (s.v[0] == 0.0) return mp_zero();
  mp x = mp_from_double(sqrt(s.v[0]));
#if ORACLE_PLANT == 4
  int steps = 0; /* planted: no Newton refinement */
#else
  int steps = (L == 1) ? 1 : (L == 2) ? 2 : (L == 4) ? 3 : 4; /* ceil(log2 L) + 1 */
#endif
  for (int it = 0; it < steps; ++it) {
    mp r = mp_sub(s, mp_mul(x, x, L), L);
    mp c = mp_half(mp_div(r, x, L), L);
    x = mp_add(x, c, L);
  }
  return x;
}

/* ---------------------------------------------------------------- complex */

static cx cx_zero(void) {
  cx z;
  memset(&z, 0, sizeof z);
  return z;
}

static cx cx_load(const double *p, int L) {
  cx z = cx_zero();
  for (int i = 0; i < L; ++i) {
    z.re.v[i] = p[i];
    z.im.v[i] = p[L + i];
  }
  return z;
}

static void cx_store(double *p, const cx *z, int L) {
  for (int i = 0; i < L; ++i) {
    p[i] = z->re.v[i];
    p[L + i] = z->im.v[i];
  }
}

static cx cx_add(cx a, cx b, int L) {
  cx z;
  z.re = mp_add(a.re, b.re, L);
  z.im = mp_add(a.im, b.im, L);
  return z;
}

static cx cx_sub(cx a, cx b, int L) {
  cx z;
  z.re = mp_sub(a.re, b.re, L);
  z.im = mp_sub(a.im, b.im, L);
  return z;
}

/* (a.re + i a.im)(b.re + i b.im) = (a.re b.re - a.im b.im) + i (a.re b.im + a.im b.re) */
static cx cx_mul(cx a, cx b, int L) {
  cx z;
  z.re = mp_sub(mp_mul(a.re, b.re, L), mp_mul(a.im, b.im, L), L);
  z.im = mp_add(mp_mul(a.re, b.im, L), mp_mul(a.im, b.re, L), L);
  return z;
}

/* conj(a) b = (a.re b.re + a.im b.im) + i (a.re b.im - a.im b.re) */
static cx cx_conjmul(cx a, cx b, int L) {
#if ORACLE_PLANT == 2
  return cx_mul(a, b, L); /* planted: the first factor is not conjugated */
#else
  cx z;
  z.re = mp_add(mp_mul(a.re, b.re, L), mp_mul(a.im, b.im, L), L);
  z.im = mp_sub(mp_mul(a.re, b.im, L), mp_mul(a.im, b.re, L), L);
  return z;
#endif
}

/* a / r for real r: two real divisions */
static cx cx_div_real(cx a, mp r, int L) {
  cx z;
  z.re = mp_div(a.re, r, L);
  z.im = mp_div(a.im, r, L);
  return z;
}

/* |a|^2 = re^2 + im^2 */
static mp cx_abs2(cx a, int L) {
#if ORACLE_PLANT == 8
  return mp_mul(a.re, a.re, L); /* planted: imaginary part left out of the norm */
#else
  return mp_add(mp_mul(a.re, a.re, L), mp_mul(a.im, a.im, L), L);
#endif
}

/* ---------------------------------------------------------------- exported primitives */

#define EXPORT __attribute__((visibility("default")))

static mp mp_load(const double *p, int L) {
  mp z = mp_zero();
  for (int i = 0; i < L; ++i) z.v[i] = p[i];
  return z;
}

static void mp_store(double *p, const mp *z, int L) {
  for (int i = 0; i < L; ++i) p[i] = z->v[i];
}

EXPORT int oracle_version(void) { return 1; }
EXPORT int oracle_plant(void) { return ORACLE_PLANT; }
EXPORT int oracle_overflowed(void) { return g_overflow; }

/* Returns 1 when the error-free transforms are exact in this build (no FMA contraction,
   round-to-nearest double arithmetic), 0 otherwise. */
EXPORT int oracle_selfcheck(void) {
  volatile double a = 1.0 + 0x1p-30, b = 1.0 - 0x1p-30;
  double p, e;
  two_prod(a, b, &p, &e);
  /* a*b = 1 - 2^-60 exactly; fl() gives 1, error -2^-60 */
  if (!(p == 1.0 && e == -0x1p-60)) return 0;
  double s, t;
  volatile double c = 0x1p60, d = 1.0;
  two_sum(c, d, &s, &t);
  if (!(s == 0x1p60 && t == 1.0)) return 0;
  /* double rounding (x87 extended registers) would break two-sum: 1 + (2^-53 + 2^-105)
     must round once, upwards, to 1 + 2^-52 */
  volatile double u = 0x1p-53 + 0x1p-105;
  double x = 1.0 + u;
  return x == 1.0 + 0x1p-52;
}

EXPORT void oracle_two_sum(double a, double b, double *s, double *e) { two_sum(a, b, s, e); }
EXPORT void oracle_two_prod(double a, double b, double *p, double *e) { two_prod(a, b, p, e); }

EXPORT void oracle_add(int L, const double *a, const double *b, double *out) {
  mp r = mp_add(mp_load(a, L), mp_load(b, L), L);
  mp_store(out, &r, L);
}
EXPORT void oracle_sub(int L, const double *a, const double *b, double *out) {
  mp r = mp_sub(mp_load(a, L), mp_load(b, L), L);
  mp_store(out, &r, L);
}
EXPORT void oracle_mul(int L, const double *a, const double *b, double *out) {
  mp r = mp_mul(mp_load(a, L), mp_load(b, L), L);
  mp_store(out, &r, L);
}
EXPORT void oracle_div(int L, const double *a, const double *b, double *out) {
  mp r = mp_div(mp_load(a, L), mp_load(b, L), L);
  mp_store(out, &r, L);
}
EXPORT void oracle_sqrt(int L, const double *a, double *out) {
  mp r = mp_sqrt(mp_load(a, L), L);
  mp_store(out, &r, L);
}
EXPORT void oracle_cmul(int L, const double *a, const double *b, double *out) {
  cx r = cx_mul(cx_load(a, L), cx_load(b, L), L);
  cx_store(out, &r, L);
}
EXPORT void oracle_cconjmul(int L, const double *a, const double *b, double *out) {
  cx r = cx_conjmul(cx_load(a, L), cx_load(b, L), L);
  cx_store(out, &r, L);
}

/* ---------------------------------------------------------------- MGS (Figure 1, Eq. 1) */

#define ELEM(base, i, j, ld, L) ((base) + ((size_t)(j) * (size_t)(ld) + (size_t)(i)) * 2 * (size_t)(L))

/*
 * Modified Gram-Schmidt on the m x nc matrix W (column-major, leading dimension ldw).
 * On return columns 0..nq-1 of W hold Q, with nq = nc - 1 when aug != 0 (the last column
 * is the right-hand side b of Eq. (1): it is reduced against q_1..q_n but not normalised,
 * so it ends as the residual vector) and nq = nc otherwise.  R (nc x nc, leading
 * dimension ldr) receives r_kj for k <= j; its diagonal is real (imaginary limbs zero).
 * When aug != 0, R[nc-1][nc-1] = z = ||residual||.  Entries below the diagonal are left
 * as they were.
 * Returns 0, or 2 when some r_kk of a column that must be normalised is zero or not
 * finite (the paper's method does not pivot, Section 4); the outputs are then
 * unspecified.
 */
EXPORT int oracle_mgs(int L, double *W, int m, int nc, int ldw, double *R, int ldr, int aug) {
  int status = 0;
  int nq = aug ? nc - 1 : nc;
  for (int k = 0; k < nc; ++k) {
    mp s = mp_zero();
    for (int l = 0; l < m; ++l) s = mp_add(s, cx_abs2(cx_load(ELEM(W, l, k, ldw, L), L), L), L);
    mp rkk = mp_sqrt(s, L);
    cx rd = cx_zero();
    rd.re = rkk;
    cx_store(ELEM(R, k, k, ldr, L), &rd, L);
    if (k >= nq) break; /* the right-hand-side column: keep z only */
    if (rkk.v[0] == 0.0 || !mp_finite(&rkk, L)) {
      status = 2;
      continue;
    }
    for (int l = 0; l < m; ++l) {
      double *p = ELEM(W, l, k, ldw, L);
      cx q = cx_div_real(cx_load(p, L), rkk, L);
      cx_store(p, &q, L);
    }
    for (int j = k + 1; j < nc; ++j) {
      cx r = cx_zero();
      for (int l = 0; l < m; ++l)
        r = cx_add(r, cx_conjmul(cx_load(ELEM(W, l, k, ldw, L), L), cx_load(ELEM(W, l, j, ldw, L), L), L), L);
      cx_store(ELEM(R, k, j, ldr, L), &r, L);
      for (int l = 0; l < m; ++l) {
        double *p = ELEM(W, l, j, ldw, L);
        cx prod = cx_mul(r, cx_load(ELEM(W, l, k, ldw, L), L), L);
#if ORACLE_PLANT == 6
        cx a = cx_add(cx_load(p, L), prod, L); /* planted: wrong sign in the update */
#else
        cx a = cx_sub(cx_load(p, L), prod, L);
#endif
        cx_store(p, &a, L);
      }
    }
  }
  if (g_overflow) status = 99;
  return status;
}

/*
 * Back substitution R x = y in the column order of Figure 3: for k = n-1..0,
 * x_k = y_k / r_kk (r_kk real: two real divisions), then y_j -= r_jk x_k for j < k.
 * y is overwritten.  Returns 0, or 2 if some r_kk is zero.
 */
EXPORT int oracle_backsub(int L, const double *R, int ldr, int n, double *y, double *x) {
  int status = 0;
  for (int k = n - 1; k >= 0; --k) {
    mp rkk = cx_load(ELEM(R, k, k, ldr, L), L).re;
    if (rkk.v[0] == 0.0) status = 2;
    cx xk = cx_div_real(cx_load(y + (size_t)k * 2 * L, L), rkk, L);
    cx_store(x + (size_t)k * 2 * L, &xk, L);
    for (int j = 0; j < k; ++j) {
#if ORACLE_PLANT == 3
      cx rjk = cx_load(ELEM(R, k, j, ldr, L), L); /* planted: transposed index */
#else
      cx rjk = cx_load(ELEM(R, j, k, ldr, L), L);
#endif
      cx yj = cx_sub(cx_load(y + (size_t)j * 2 * L, L), cx_mul(rjk, xk, L), L);
      cx_store(y + (size_t)j * 2 * L, &yj, L);
    }
  }
  return status;
}

/*
 * Least squares min ||b - A x|| through MGS on [A b] (Eq. 1) and Figure 3.
 *   A: m x n, lda; on return holds Q.        b: m; on return holds the residual b - A x.
 *   x: n (out).   R: n x n, ldr (out; may be NULL).   z: L limbs (out; may be NULL).
 * Returns 0, 1 for bad sizes, 2 for a zero/non-finite r_kk.
 */
EXPORT int oracle_ls_solve(int L, double *A, double *b, double *x, double *R, double *z, int m, int n, int lda,
                           int ldr) {
  if (L != 1 && L != 2 && L != 4 && L != 8) return 1;
  if (n < 1 || m < n || lda < m) return 1;
  int nc = n + 1;
  size_t es = 2 * (size_t)L;
  double *W = (double *)malloc(sizeof(double) * es * (size_t)m * nc);
  double *Rw = (double *)calloc(es * (size_t)nc * nc, sizeof(double));
  double *yv = (double *)malloc(sizeof(double) * es * (size_t)n);
  if (!W || !Rw || !yv) {
    free(W);
    free(Rw);
    free(yv);
    return 1;
  }
  for (int j = 0; j < n; ++j) memcpy(ELEM(W, 0, j, m, L), ELEM(A, 0, j, lda, L), sizeof(double) * es * m);
  memcpy(ELEM(W, 0, n, m, L), b, sizeof(double) * es * m);
  int st = oracle_mgs(L, W, m, nc, m, Rw, nc, 1);
  for (int j = 0; j < n; ++j) memcpy(ELEM(A, 0, j, lda, L), ELEM(W, 0, j, m, L), sizeof(double) * es * m);
  memcpy(b, ELEM(W, 0, n, m, L), sizeof(double) * es * m);
  for (int k = 0; k < n; ++k) memcpy(yv + k * es, ELEM(Rw, k, n, nc, L), sizeof(double) * es);
  if (R)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k <= j; ++k) memcpy(ELEM(R, k, j, ldr, L), ELEM(Rw, k, j, nc, L), sizeof(double) * es);
  if (z) memcpy(z, ELEM(Rw, n, n, nc, L), sizeof(double) * L);
  int st2 = oracle_backsub(L, Rw, nc, n, yv, x);
  free(W);
  free(Rw);
  free(yv);
  if (st) return st;
  return st2;
}

/* QR only (Figure 1 without the augmented column): A (m x n) -> Q in place, R (n x n). */
EXPORT int oracle_qr(int L, double *A, double *R, int m, int n, int lda, int ldr) {
  if (L != 1 && L != 2 && L != 4 && L != 8) return 1;
  if (n < 1 || m < n || lda < m || ldr < n) return 1;
  return oracle_mgs(L, A, m, n, lda, R, ldr, 0);
}

/* ---------------------------------------------------------------- exact checks */

static double xp_to_double(xp *E) {
  xp_compress(E);
  return xp_approx(E);
}

/*
 * b = A x with every entry summed exactly and rounded once to Lout limbs
 * (A and x carry Lin limbs).  Used to plant a solution x_true in b = A x_true.
 */
EXPORT void oracle_matvec(int Lin, const double *A, int m, int n, int lda, const double *x, int Lout, double *b) {
  static __thread xp Er, Ei;
  for (int i = 0; i < m; ++i) {
    Er.n = 0;
    Ei.n = 0;
    for (int j = 0; j < n; ++j) {
      cx a = cx_load(ELEM(A, i, j, lda, Lin), Lin);
      cx v = cx_load(x + (size_t)j * 2 * Lin, Lin);
      xp_add_prod(&Er, &a.re, &v.re, Lin, 1.0);
#if ORACLE_PLANT == 10
      xp_add_prod(&Er, &a.im, &v.im, Lin, 1.0); /* planted: wrong sign of the im*im term */
#else
      xp_add_prod(&Er, &a.im, &v.im, Lin, -1.0);
#endif
      xp_add_prod(&Ei, &a.re, &v.im, Lin, 1.0);
      xp_add_prod(&Ei, &a.im, &v.re, Lin, 1.0);
      if (Er.n > 256) xp_compress(&Er);
      if (Ei.n > 256) xp_compress(&Ei);
    }
    cx z;
    z.re = xp_round(&Er, Lout);
    z.im = xp_round(&Ei, Lout);
    cx_store(b + (size_t)i * 2 * Lout, &z, Lout);
  }
}

/*
 * out = A^H v (n entries): out_j = sum_i conj(a_ij) v_i, each sum exact, then rounded to
 * Lout limbs.  conj(a) v = (ar vr + ai vi) + i (ar vi - ai vr).  With v a column of Q this
 * is a column of Q^H Q (the orthogonality of Section 3); with v = b - A x it is the
 * normal-equations residual of the least-squares solution.
 */
EXPORT void oracle_matvec_conjT(int Lin, const double *A, int m, int n, int lda, const double *v, int Lout,
                                double *out) {
  static __thread xp Er, Ei;
  for (int j = 0; j < n; ++j) {
    Er.n = 0;
    Ei.n = 0;
    for (int i = 0; i < m; ++i) {
      cx a = cx_load(ELEM(A, i, j, lda, Lin), Lin);
      cx w = cx_load(v + (size_t)i * 2 * Lin, Lin);
      xp_add_prod(&Er, &a.re, &w.re, Lin, 1.0);
#if ORACLE_PLANT == 9
      xp_add_prod(&Er, &a.im, &w.im, Lin, -1.0); /* planted: A^T v instead of A^H v */
#else
      xp_add_prod(&Er, &a.im, &w.im, Lin, 1.0);
#endif
      xp_add_prod(&Ei, &a.re, &w.im, Lin, 1.0);
      xp_add_prod(&Ei, &a.im, &w.re, Lin, -1.0);
      if (Er.n > 256) xp_compress(&Er);
      if (Ei.n > 256) xp_compress(&Ei);
    }
    cx z;
    z.re = xp_round(&Er, Lout);
    z.im = xp_round(&Ei, Lout);
    cx_store(out + (size_t)j * 2 * Lout, &z, Lout);
  }
}

/*
 * Eq. (2): e = max_{i,j} | a_ij - sum_l q_il r_lj | (complex modulus), the inner sum and
 * the difference evaluated exactly, the modulus in double.  A is the ORIGINAL matrix,
 * Q (m x n) and R (n x n, upper) the computed factors; all carry L limbs.
 * Also returns in *emax_part the max over real and imaginary parts separately.
 */
EXPORT double oracle_qr_error(int L, const double *A, int lda, const double *Q, int ldq, const double *R, int ldr,
                              int m, int n, double *emax_part) {
  static __thread xp Er, Ei;
  double emax = 0.0, epart = 0.0;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < m; ++i) {
      Er.n = 0;
      Ei.n = 0;
      cx a = cx_load(ELEM(A, i, j, lda, L), L);
      xp_add_mp(&Er, &a.re, L, 1.0);
      xp_add_mp(&Ei, &a.im, L, 1.0);
      for (int l = 0; l <= j; ++l) {
        cx q = cx_load(ELEM(Q, i, l, ldq, L), L);
        cx r = cx_load(ELEM(R, l, j, ldr, L), L);
        xp_add_prod(&Er, &q.re, &r.re, L, -1.0);
        xp_add_prod(&Er, &q.im, &r.im, L, 1.0);
        xp_add_prod(&Ei, &q.re, &r.im, L, -1.0);
        xp_add_prod(&Ei, &q.im, &r.re, L, -1.0);
        if (Er.n > 256) xp_compress(&Er);
        if (Ei.n > 256) xp_compress(&Ei);
      }
      double dr = xp_to_double(&Er), di = xp_to_double(&Ei);
      double e = hypot(dr, di);
      if (e > emax) emax = e;
      if (fabs(dr) > epart) epart = fabs(dr);
      if (fabs(di) > epart) epart = fabs(di);
    }
  if (emax_part) *emax_part = epart;
  return emax;
}

/* max_{i,j} | (Q^H Q - I)_ij |, inner products exact, modulus in double. */
EXPORT double oracle_orth_error(int L, const double *Q, int ldq, int m, int n) {
  static __thread xp Er, Ei;
  double emax = 0.0;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      Er.n = 0;
      Ei.n = 0;
      if (i == j) xp_grow(&Er, -1.0);
      for (int l = 0; l < m; ++l) {
        cx a = cx_load(ELEM(Q, l, i, ldq, L), L);
        cx b = cx_load(ELEM(Q, l, j, ldq, L), L);
        /* conj(a) b */
        xp_add_prod(&Er, &a.re, &b.re, L, 1.0);
        xp_add_prod(&Er, &a.im, &b.im, L, 1.0);
        xp_add_prod(&Ei, &a.re, &b.im, L, 1.0);
        xp_add_prod(&Ei, &a.im, &b.re, L, -1.0);
        if (Er.n > 256) xp_compress(&Er);
        if (Ei.n > 256) xp_compress(&Ei);
      }
      double e = hypot(xp_to_double(&Er), xp_to_double(&Ei));
      if (e > emax) emax = e;
    }
  return emax;
}

/*
 * Residual vector r = b - A x, each entry exact then rounded to Lout limbs, and
 * ||r||_2^2 exactly (returned as a double approximation).  A, b, x carry L limbs.
 */
EXPORT double oracle_residual(int L, const double *A, int lda, const double *b, const double *x, int m, int n,
                              int Lout, double *r_out) {
  static __thread xp Er, Ei, N2;
  N2.n = 0;
  for (int i = 0; i < m; ++i) {
    Er.n = 0;
    Ei.n = 0;
    cx bi = cx_load(b + (size_t)i * 2 * L, L);
    xp_add_mp(&Er, &bi.re, L, 1.0);
    xp_add_mp(&Ei, &bi.im, L, 1.0);
    for (int j = 0; j < n; ++j) {
      cx a = cx_load(ELEM(A, i, j, lda, L), L);
      cx v = cx_load(x + (size_t)j * 2 * L, L);
      xp_add_prod(&Er, &a.re, &v.re, L, -1.0);
      xp_add_prod(&Er, &a.im, &v.im, L, 1.0);
      xp_add_prod(&Ei, &a.re, &v.im, L, -1.0);
      xp_add_prod(&Ei, &a.im, &v.re, L, -1.0);
      if (Er.n > 256) xp_compress(&Er);
      if (Ei.n > 256) xp_compress(&Ei);
    }
    cx z;
    xp_compress(&Er);
    xp_compress(&Ei);
    z.re = xp_round(&Er, 4);
    z.im = xp_round(&Ei, 4);
    if (r_out) {
      for (int t = 0; t < Lout; ++t) {
        r_out[(size_t)i * 2 * Lout + t] = z.re.v[t];
        r_out[(size_t)i * 2 * Lout + Lout + t] = z.im.v[t];
      }
    }
    /* ||r||^2 accumulates |r_i|^2 of the 4-limb rounded entries (relative 2^-200) */
    xp_add_prod(&N2, &z.re, &z.re, 4, 1.0);
    xp_add_prod(&N2, &z.im, &z.im, 4, 1.0);
    if (N2.n > 256) xp_compress(&N2);
  }
  return xp_to_double(&N2);
}

/*
 * ||R^{-1}||_F for the upper-triangular R (n x n, ldr), by solving R X = I column by
 * column with back substitution in L-limb arithmetic; used for the condition estimate
 * kappa = ||A||_F ||R^{-1}||_F.  Returns -1 when some r_kk is zero.
 */
EXPORT double oracle_rinv_fro(int L, const double *R, int ldr, int n) {
  size_t es = 2 * (size_t)L;
  double *y = (double *)calloc(es * (size_t)n, sizeof(double));
  double *x = (double *)calloc(es * (size_t)n, sizeof(double));
  if (!y || !x) {
    free(y);
    free(x);
    return -1.0;
  }
  double acc = 0.0;
  int bad = 0;
  for (int c = 0; c < n; ++c) {
    memset(y, 0, sizeof(double) * es * n);
    y[(size_t)c * es] = 1.0;
    /* only rows 0..c are nonzero in column c of R^{-1} */
    if (oracle_backsub(L, R, ldr, c + 1, y, x)) bad = 1;
    for (int k = 0; k <= c; ++k) {
      cx v = cx_load(x + k * es, L);
      double re = mp_approx(&v.re, L);
      double im = mp_approx(&v.im, L);
      acc += re * re + im * im;
    }
  }
  free(y);
  free(x);
  return bad ? -1.0 : sqrt(acc);
}

/*
 * Exact comparison helper: for count complex elements a_i (La limbs) and b_i (Lb limbs),
 * returns max_i |a_i - b_i| (difference exact, modulus in double) and, in *max_abs_b,
 * max_i |b_i|.
 */
EXPORT double oracle_max_abs_diff(int La, const double *a, int Lb, const double *b, long count, double *max_abs_b) {
  static __thread xp Er, Ei;
  double dmax = 0.0, bmax = 0.0;
  for (long i = 0; i < count; ++i) {
    cx x = cx_load(a + (size_t)i * 2 * La, La);
    cx y = cx_load(b + (size_t)i * 2 * Lb, Lb);
    Er.n = 0;
    Ei.n = 0;
    xp_add_mp(&Er, &x.re, La, 1.0);
    xp_add_mp(&Ei, &x.im, La, 1.0);
    xp_add_mp(&Er, &y.re, Lb, -1.0);
    xp_add_mp(&Ei, &y.im, Lb, -1.0);
    double d = hypot(xp_to_double(&Er), xp_to_double(&Ei));
    double bb = hypot(mp_approx(&y.re, Lb), mp_approx(&y.im, Lb));
    if (d > dmax || d != d) dmax = d;
    if (bb > bmax) bmax = bb;
  }
  if (max_abs_b) *max_abs_b = bmax;
  return dmax;
}

/* ---------------------------------------------------------------- adjoint of least squares */

/*
 * Forward substitution with the conjugate transpose: R^H u = g (R upper triangular with
 * real diagonal), column order: for k = 0..n-1, u_k = g_k / r_kk, then
 * g_j -= conj(r_kj) u_k for j > k.  g is overwritten.
 */
EXPORT int oracle_fwdsub_conjT(int L, const double *R, int ldr, int n, double *g, double *u) {
  int status = 0;
  for (int k = 0; k < n; ++k) {
    mp rkk = cx_load(ELEM(R, k, k, ldr, L), L).re;
    if (rkk.v[0] == 0.0) status = 2;
    cx uk = cx_div_real(cx_load(g + (size_t)k * 2 * L, L), rkk, L);
    cx_store(u + (size_t)k * 2 * L, &uk, L);
    for (int j = k + 1; j < n; ++j) {
      cx rkj = cx_load(ELEM(R, k, j, ldr, L), L);
      cx gj = cx_sub(cx_load(g + (size_t)j * 2 * L, L), cx_conjmul(rkj, uk, L), L);
      cx_store(g + (size_t)j * 2 * L, &gj, L);
    }
  }
  return status;
}

/*
 * Adjoint of x = argmin ||b - A x|| for a real loss L(x) with gradient G = dL/dRe(x) +
 * i dL/dIm(x): from A^H A x = A^H b,
 *     w = (A^H A)^{-1} G = R^{-1} R^{-H} G,   grad_b = A w = Q R^{-H} G,
 *     grad_A = r w^H - grad_b x^H,             r = b - A x,
 * with Q, R, x, r from MGS on [A b] (Eq. 1) and Figure 3.  Every product of grad_A is
 * formed exactly and rounded once.  A (m x n) and b are the original inputs.
 * Returns 0, or the status of the solve.
 */
EXPORT int oracle_ls_adjoint(int L, const double *A, const double *b, const double *G, int m, int n, double *gA,
                             double *gb, double *x_out) {
  size_t es = 2 * (size_t)L;
  double *Q = (double *)malloc(sizeof(double) * es * (size_t)m * n);
  double *r = (double *)malloc(sizeof(double) * es * (size_t)m);
  double *R = (double *)calloc(es * (size_t)n * n, sizeof(double));
  double *x = (double *)malloc(sizeof(double) * es * (size_t)n);
  double *g = (double *)malloc(sizeof(double) * es * (size_t)n);
  double *u = (double *)malloc(sizeof(double) * es * (size_t)n);
  double *w = (double *)malloc(sizeof(double) * es * (size_t)n);
  if (!Q || !r || !R || !x || !g || !u || !w) return 1;
  memcpy(Q, A, sizeof(double) * es * m * n);
  memcpy(r, b, sizeof(double) * es * m);
  int st = oracle_ls_solve(L, Q, r, x, R, NULL, m, n, m, n);
  memcpy(g, G, sizeof(double) * es * n);
  st |= oracle_fwdsub_conjT(L, R, n, n, g, u);  /* u = R^{-H} G */
  memcpy(g, u, sizeof(double) * es * n);
  st |= oracle_backsub(L, R, n, n, g, w);        /* w = R^{-1} u */
  oracle_matvec(L, Q, m, n, m, u, L, gb);        /* grad_b = Q u */
  static __thread xp Er, Ei;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < m; ++i) {
      cx ri = cx_load(r + (size_t)i * es, L), wj = cx_load(w + (size_t)j * es, L);
      cx gi = cx_load(gb + (size_t)i * es, L), xj = cx_load(x + (size_t)j * es, L);
      Er.n = 0;
      Ei.n = 0;
      /* r_i conj(w_j) = (rr wr + ri wi) + i (ri wr - rr wi) */
      xp_add_prod(&Er, &ri.re, &wj.re, L, 1.0);
      xp_add_prod(&Er, &ri.im, &wj.im, L, 1.0);
      xp_add_prod(&Ei, &ri.im, &wj.re, L, 1.0);
      xp_add_prod(&Ei, &ri.re, &wj.im, L, -1.0);
      /* - g_i conj(x_j) */
      xp_add_prod(&Er, &gi.re, &xj.re, L, -1.0);
#if ORACLE_PLANT == 11
      xp_add_prod(&Er, &gi.im, &xj.im, L, 1.0); /* planted: g_i x_j^T instead of g_i x_j^H */
#else
      xp_add_prod(&Er, &gi.im, &xj.im, L, -1.0);
#endif
      xp_add_prod(&Ei, &gi.im, &xj.re, L, -1.0);
      xp_add_prod(&Ei, &gi.re, &xj.im, L, 1.0);
      cx o;
      o.re = xp_round(&Er, L);
      o.im = xp_round(&Ei, L);
      cx_store(ELEM(gA, i, j, m, L), &o, L);
    }
  if (x_out) memcpy(x_out, x, sizeof(double) * es * n);
  free(Q);
  free(r);
  free(R);
  free(x);
  free(g);
  free(u);
  free(w);
  return st;
}
