"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each ``pin_*`` function raises AssertionError when the oracle it is given is wrong.  The
test modules run them on the real oracle; ``test_oracle_plants`` runs them on oracle builds
with a planted mistake and requires every plant to be caught by at least one pin.

Exact references are Python ``fractions.Fraction`` values: every double is a dyadic
rational, so sums, products and quotients of limb values are computed without rounding.
"""

from __future__ import annotations

import math
import os
from fractions import Fraction as F

import numpy as np

from paper_1210_0800_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ----------------------------------------------------------------------------- helpers


def fval(limbs) -> F:
    """Exact value of a limb vector."""
    return sum((F(float(v)) for v in np.ravel(limbs)), F(0))


def cval(elem):
    """Exact (re, im) of a complex element of shape (2, L)."""
    e = np.asarray(elem).reshape(2, -1)
    return fval(e[0]), fval(e[1])


def cabs2(z) -> F:
    return z[0] * z[0] + z[1] * z[1]


def cmul(a, b):
    return (a[0] * b[0] - a[1] * b[1], a[0] * b[1] + a[1] * b[0])


def cconj(a):
    return (a[0], -a[1])


def csub(a, b):
    return (a[0] - b[0], a[1] - b[1])


def cadd(a, b):
    return (a[0] + b[0], a[1] + b[1])


def cdiv(a, b):
    d = cabs2(b)
    n = cmul(a, cconj(b))
    return (n[0] / d, n[1] / d)


def cdot(x, y):
    """x^H y over lists of exact complex pairs."""
    s = (F(0), F(0))
    for a, b in zip(x, y):
        s = cadd(s, cmul(cconj(a), b))
    return s


def cnorm_inf(z) -> float:
    return math.hypot(float(z[0]), float(z[1]))


def rand_limbs(L: int, seed: int, count: int, exp_range=(-40, 40)) -> np.ndarray:
    """count random L-limb reals with leading limbs spread over 2^exp_range."""
    lead = inputs.uniform_pm1(inputs.substream(seed, 1), count)
    ex = inputs.uniform_int(inputs.substream(seed, 2), count, exp_range[0], exp_range[1])
    lead = np.ldexp(lead, ex)
    return inputs.with_lower_limbs(lead, L, inputs.substream(seed, 3))


def adversarial_pairs(L: int):
    """Operand pairs with cancellation, large exponent gaps, zeros and exact cases."""
    one = np.zeros(L)
    one[0] = 1.0
    x = rand_limbs(L, 99, 1)[0]
    pairs = [
        (x, -x),                                   # exact cancellation
        (one, np.array([2.0 ** -150] + [0.0] * (L - 1))),  # wide exponent gap
        (np.zeros(L), x),                          # zero operand
        (x, x),                                    # doubling
        (one, -one),
        (np.array([1.0, 2.0 ** -60] + [0.0] * (L - 2))[:L] if L > 1 else one,
         np.array([-1.0, 2.0 ** -70] + [0.0] * (L - 2))[:L] if L > 1 else -one),
        (np.array([3.0] + [0.0] * (L - 1)), np.array([1.0 / 3.0] + [0.0] * (L - 1))),
        (np.array([2.0 ** 40] + [0.0] * (L - 1)), np.array([-(2.0 ** 40) + 1.0] + [0.0] * (L - 1))),
    ]
    if L > 1:
        y = x.copy()
        y[-1] = -y[-1] if y[-1] != 0 else 2.0 ** -200
        pairs.append((x, -y))                      # cancellation down to the last limb
    return pairs


def u_of(L: int) -> float:
    return 2.0 ** (-53 * L)


# ----------------------------------------------------------------------------- primitives


def pin_error_free_transforms(o):
    """two_sum and two_prod are exact (Knuth; Dekker / FMA)."""
    import ctypes

    vals = list(np.ldexp(inputs.uniform_pm1(5, 400), inputs.uniform_int(6, 400, -60, 60)))
    for a, b in zip(vals[::2], vals[1::2]):
        s, e = ctypes.c_double(), ctypes.c_double()
        o.lib.oracle_two_sum(a, b, ctypes.byref(s), ctypes.byref(e))
        assert F(s.value) + F(e.value) == F(a) + F(b), ("two_sum", a, b)
        assert s.value == a + b
        o.lib.oracle_two_prod(a, b, ctypes.byref(s), ctypes.byref(e))
        assert F(s.value) + F(e.value) == F(a) * F(b), ("two_prod", a, b)
        assert s.value == a * b


def pin_real_ops(o, L: int, trials: int = 150):
    """+, -, *, / and sqrt at L limbs against exact rationals, random and adversarial
    operands; the bound is a few units of 2^(-53 L) relative to the exact result."""
    u = u_of(L)
    A = rand_limbs(L, 1000 + L, trials)
    B = rand_limbs(L, 2000 + L, trials)
    pairs = list(zip(A, B)) + adversarial_pairs(L)
    for a, b in pairs:
        fa, fb = fval(a), fval(b)
        for name, fn, exact, c in (
            ("add", o.add, fa + fb, 2),
            ("sub", o.sub, fa - fb, 2),
            ("mul", o.mul, fa * fb, 2),
        ):
            r = fval(fn(L, a, b))
            assert abs(r - exact) <= c * u * abs(exact), (name, L, a, b, float(r - exact))
        if fb != 0:
            q = fval(o.div(L, a, b))
            exact = fa / fb
            assert abs(q - exact) <= 4 * u * abs(exact), ("div", L, a, b, float(q - exact))
    for a in list(A) + [np.array([4.0] + [0.0] * (L - 1)), np.array([2.0] + [0.0] * (L - 1)), np.zeros(L)]:
        s = abs(fval(a))
        sv = np.array(a, dtype=np.float64)
        if sv[0] < 0:
            sv = -sv
        r = fval(o.sqrt(L, sv))
        if s == 0:
            assert r == 0
            continue
        assert r > 0
        assert abs(r * r - s) <= 8 * u * s, ("sqrt", L, sv, float((r * r - s) / s))
    # exact cases stay exact
    four = np.array([4.0] + [0.0] * (L - 1))
    assert fval(o.sqrt(L, four)) == 2


def pin_complex_ops(o, L: int, trials: int = 60):
    """Complex product and conjugated product (x^H y convention, Section 3) against exact
    rationals."""
    u = u_of(L)
    A = rand_limbs(L, 3000 + L, 2 * trials).reshape(trials, 2, L)
    B = rand_limbs(L, 4000 + L, 2 * trials).reshape(trials, 2, L)
    for a, b in zip(A, B):
        ca, cb = cval(a), cval(b)
        scale = math.sqrt(float(cabs2(ca))) * math.sqrt(float(cabs2(cb)))
        for fn, exact in ((o.cmul, cmul(ca, cb)), (o.cconjmul, cmul(cconj(ca), cb))):
            r = cval(fn(L, a, b))
            err = cnorm_inf(csub(r, exact))
            assert err <= 6 * u * scale, (fn.__name__, L, err / scale)


# ----------------------------------------------------------------------------- MGS


def gaussian_int_matrix(m: int, n: int, seed: int, lo=-4, hi=4) -> np.ndarray:
    vals = inputs.uniform_int(seed, 2 * m * n, lo, hi).astype(np.float64).reshape(n, m, 2)
    return vals


def embed(vals: np.ndarray, L: int) -> np.ndarray:
    out = np.zeros(vals.shape + (L,))
    out[..., 0] = vals
    return out


def exact_cgs(Aex):
    """Unnormalised Gram-Schmidt in exact arithmetic (equal to MGS in exact arithmetic):
    v_k = a_k - sum_{i<k} (v_i^H a_k / v_i^H v_i) v_i.  Returns v (list of columns)."""
    n = len(Aex)
    vs = []
    for k in range(n):
        v = list(Aex[k])
        for i in range(k):
            c = cdiv(cdot(vs[i], Aex[k]), (cdot(vs[i], vs[i])[0], F(0)))
            v = [csub(vl, cmul(c, vil)) for vl, vil in zip(v, vs[i])]
        vs.append(v)
    return vs


def exact_ls(Aex, bex):
    """Exact least-squares solution of min ||b - A x|| via the normal equations
    (A^H A) x = A^H b, solved by Gaussian elimination over the Gaussian rationals."""
    n = len(Aex)
    G = [[cdot(Aex[i], Aex[j]) for j in range(n)] for i in range(n)]
    h = [cdot(Aex[i], bex) for i in range(n)]
    M = [row[:] + [h[i]] for i, row in enumerate(G)]
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != (0, 0))
        M[c], M[p] = M[p], M[c]
        for r in range(n):
            if r != c and M[r][c] != (0, 0):
                f = cdiv(M[r][c], M[c][c])
                M[r] = [csub(M[r][k], cmul(f, M[c][k])) for k in range(n + 1)]
    return [cdiv(M[i][n], M[i][i]) for i in range(n)]


def _cols(Q):
    """(n, m, 2, L) array -> list of columns of exact complex pairs."""
    return [[cval(Q[j, i]) for i in range(Q.shape[1])] for j in range(Q.shape[0])]


def pin_mgs_exact_rational(o, L: int, cases=((1, 1), (3, 2), (4, 4), (6, 3), (5, 5), (6, 4))):
    """Tiny Gaussian-integer systems against exact rational arithmetic.  With v_k the
    unnormalised Gram-Schmidt vectors: r_kk^2 = v_k^H v_k, r_kk r_kj = v_k^H a_j,
    r_kk q_k = v_k; x solves the normal equations; z^2 = ||b - A x||^2; the reduced last
    column equals b - A x (Section 3, Figure 1 and Eq. 1)."""
    tol = u_of(L) * 2.0 ** 16
    for ci, (m, n) in enumerate(cases):
        for rep in range(2):
            seed = 500 + 37 * ci + rep
            vals = gaussian_int_matrix(m, n, seed)
            A = embed(vals, L)
            if rep == 0:
                # consistent system b = A x_true with a Gaussian-integer x_true (exact in float64)
                xt = inputs.uniform_int(seed + 1, 2 * n, -3, 3).astype(np.float64).reshape(n, 2)
                Ac = vals[..., 0] + 1j * vals[..., 1]
                bc = (Ac.T @ (xt[:, 0] + 1j * xt[:, 1]))
                bvals = np.stack([bc.real, bc.imag], axis=-1)
            else:
                # generic right-hand side (inconsistent when m > n)
                bvals = inputs.uniform_int(seed + 1, 2 * m, -5, 5).astype(np.float64).reshape(m, 2)
            b = embed(bvals, L)
            Aex = _cols(A)
            bex = [cval(b[i]) for i in range(m)]
            vs = exact_cgs(Aex)
            if any(cdot(v, v)[0] == 0 for v in vs):
                continue  # rank deficient draw: not a pin case
            res = o.ls_solve(A, b)
            assert res["status"] == 0
            R, Q = res["R"], res["Q"]
            scaleA = max(float(cabs2(a)) for col in Aex for a in col)
            for k in range(n):
                rkk = cval(R[k, k])
                assert rkk[1] == 0 and rkk[0] > 0
                vv = cdot(vs[k], vs[k])[0]
                assert abs(rkk[0] * rkk[0] - vv) <= tol * scaleA * m, ("r_kk^2", L, m, n, k)
                for i in range(m):
                    rq = (rkk[0] * cval(Q[k, i])[0], rkk[0] * cval(Q[k, i])[1])
                    assert cnorm_inf(csub(rq, vs[k][i])) <= tol * math.sqrt(scaleA) * m, ("r_kk q_k", L, m, n, k)
                for j in range(k + 1, n):
                    prod = (rkk[0] * cval(R[j, k])[0], rkk[0] * cval(R[j, k])[1])
                    assert cnorm_inf(csub(prod, cdot(vs[k], Aex[j]))) <= tol * scaleA * m, ("r_kk r_kj", L, k, j)
            xex = exact_ls(Aex, bex)
            xs = [cval(res["x"][k]) for k in range(n)]
            xscale = max(max(cnorm_inf(v) for v in xex), 1.0)
            for k in range(n):
                assert cnorm_inf(csub(xs[k], xex[k])) <= tol * 64 * xscale, ("x", L, m, n, k)
            # residual column and z (Eq. 1): reduced b equals b - A x_exact, z = its norm
            rex = [csub(bex[i], sum_cols(Aex, xex, i)) for i in range(m)]
            bscale = max(max(cnorm_inf(v) for v in bex), 1.0)
            for i in range(m):
                assert cnorm_inf(csub(cval(res["resid"][i]), rex[i])) <= tol * 64 * bscale, ("resid", L, i)
            z = fval(res["z"])
            z2 = sum(cabs2(r) for r in rex)
            assert abs(z * z - z2) <= tol * 64 * bscale * bscale * m, ("z", L, m, n, float(z * z), float(z2))


def sum_cols(Aex, x, i):
    s = (F(0), F(0))
    for j in range(len(Aex)):
        s = cadd(s, cmul(Aex[j][i], x[j]))
    return s


def pin_mgs_special_cases(o, L: int):
    """Special cases with a closed form.
    (a) n = 1: r_11 = ||a||, x = a^H b / ||a||^2.
    (b) the 4 x 4 Fourier matrix F_jk = i^{jk}: orthogonal columns of norm 2, so MGS gives
        R = 2 I and Q = F / 2 exactly.
    (c) upper-triangular A with positive real diagonal (m = n): Q = I and R = A exactly.
    (d) A = P D (permutation times complex diagonal): R diagonal with |d_k|."""
    u = u_of(L)
    # (a)
    a = embed(np.array([[[3.0, 4.0], [0.0, -2.0], [1.0, 1.0]]]), L)  # one column, m = 3
    b = embed(np.array([[1.0, 0.0], [2.0, -1.0], [0.0, 3.0]]), L)
    res = o.ls_solve(a, b)
    aex = _cols(a)[0]
    bex = [cval(b[i]) for i in range(3)]
    nrm2 = cdot(aex, aex)[0]
    xex = cdiv(cdot(aex, bex), (nrm2, F(0)))
    r11 = fval(res["R"][0, 0, 0])
    assert abs(r11 * r11 - nrm2) <= 8 * u * nrm2
    assert cnorm_inf(csub(cval(res["x"][0]), xex)) <= 64 * u * cnorm_inf(xex)
    # (b)
    Fm = np.zeros((4, 4, 2))
    for j in range(4):
        for k in range(4):
            ph = (j * k) % 4
            Fm[k, j] = [(1, 0), (0, 1), (-1, 0), (0, -1)][ph]  # column k, row j
    Q, R, st = o.qr(embed(Fm, L))
    assert st == 0
    for j in range(4):
        for k in range(4):
            want = (F(2), F(0)) if j == k else (F(0), F(0))
            if k <= j:
                assert cval(R[j, k]) == want, ("DFT R", j, k)
            assert cval(Q[k, j]) == (F(Fm[k, j, 0]) / 2, F(Fm[k, j, 1]) / 2), ("DFT Q", j, k)
    # (c)
    n = 5
    T = np.zeros((n, n, 2))
    tv = gaussian_int_matrix(n, n, 77)
    for j in range(n):
        for i in range(j + 1):
            T[j, i] = tv[j, i]
        T[j, j] = [float(j + 2), 0.0]
    Q, R, st = o.qr(embed(T, L))
    assert st == 0
    for j in range(n):
        for i in range(n):
            assert cval(Q[j, i]) == ((F(1) if i == j else F(0)), F(0)), ("triangular Q", i, j)
            if i <= j:
                assert cval(R[j, i]) == (F(T[j, i, 0]), F(T[j, i, 1])), ("triangular R", i, j)
    # (d)
    perm = [2, 0, 3, 1]
    d = [(3.0, 4.0), (0.0, -2.0), (5.0, 12.0), (-1.0, 0.0)]
    Pm = np.zeros((4, 4, 2))
    for k in range(4):
        Pm[k, perm[k]] = d[k]
    Q, R, st = o.qr(embed(Pm, L))
    assert st == 0
    mods = [5.0, 2.0, 13.0, 1.0]
    for j in range(4):
        for k in range(j + 1):
            want = (F(mods[j]), F(0)) if j == k else (F(0), F(0))
            assert cnorm_inf(csub(cval(R[j, k]), want)) <= 8 * u * mods[j], ("perm R", j, k)
        q = cval(Q[j, perm[j]])
        want = (F(d[j][0]) / F(mods[j]), F(d[j][1]) / F(mods[j]))
        assert cnorm_inf(csub(q, want)) <= 8 * u, ("perm Q", j)


def pin_backsub(o, L: int, n: int = 6):
    """Figure 3 solves R x = y: the exact residual R x - y is at rounding level (a
    transposed R would not solve the system)."""
    u = u_of(L)
    vals = gaussian_int_matrix(n, n, 4242, -9, 9)
    R = np.zeros((n, n, 2))
    for j in range(n):
        for i in range(j + 1):
            R[j, i] = vals[j, i]
        R[j, j] = [float(3 + j), 0.0]
    y = inputs.uniform_int(4343, 2 * n, -9, 9).astype(np.float64).reshape(n, 2)
    x, st = o.backsub(embed(R, L), embed(y, L))
    assert st == 0
    xs = [cval(x[k]) for k in range(n)]
    for i in range(n):
        s = (F(0), F(0))
        for k in range(i, n):
            s = cadd(s, cmul((F(R[k, i, 0]), F(R[k, i, 1])), xs[k]))
        err = cnorm_inf(csub(s, (F(y[i, 0]), F(y[i, 1]))))
        assert err <= 2.0 ** 12 * u * 10, ("backsub residual", L, i, err)


def load_table2():
    rows = {}
    with open(os.path.join(GOLDEN, "table2_accuracy.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            p, g, lo, hi = line.split()
            rows[(p, int(g))] = (float(lo), float(hi))
    return rows


PREC_L = {"D": 1, "DD": 2, "QD": 4}


def table2_logs(o, prec: str, g: int, count: int, seed0: int = 777000):
    L = PREC_L[prec]
    logs = []
    for s in range(count):
        A = inputs.complex_polar((32, 32), L, seed0 + s, g)
        Q, R, st = o.qr(A)
        assert st == 0
        e, _ = o.qr_error(A, Q, R)
        logs.append(math.log10(e))
    return logs


def pin_table2(o, prec: str, g: int, count: int, margin: float = 0.5):
    """Table 2 (Section 4): log10 e of 32 x 32 QR decompositions of the paper's random
    matrices lies inside the printed [m_e, M_e] widened by ``margin`` decades."""
    lo, hi = load_table2()[(prec, g)]
    logs = table2_logs(o, prec, g, count)
    assert min(logs) >= lo - margin and max(logs) <= hi + margin, (prec, g, min(logs), max(logs), lo, hi)
    return logs


def pin_matvec(o, L: int, Lout: int):
    """A x and A^H v against exact rational arithmetic: every entry within one rounding to
    Lout limbs of the exact sum (one row of v is itself a combination of A's columns, so
    the sums cancel)."""
    m, n = 7, 5
    A = inputs.matrix_uniform(m, n, L, 6101)
    x = inputs.system(m, n, L, 6102)[1]
    v = inputs.system(m, n, L, 6103)[2]
    v[3] = o.matvec(A, x)[3]
    Aex = [[cval(A[j, i]) for j in range(n)] for i in range(m)]
    xex = [cval(x[j]) for j in range(n)]
    vex = [cval(v[i]) for i in range(m)]
    got = o.matvec(A, x, Lout=Lout)
    gotT = o.matvec_conjT(A, v, Lout=Lout)
    u = 2.0 ** (-53 * Lout)
    for i in range(m):
        want = (sum((cmul(Aex[i][j], xex[j])[0] for j in range(n)), F(0)),
                sum((cmul(Aex[i][j], xex[j])[1] for j in range(n)), F(0)))
        g = cval(got[i])
        for p in range(2):
            assert abs(float(g[p] - want[p])) <= 2 * u * abs(float(want[p])) + 1e-300
    for j in range(n):
        want = cdot([Aex[i][j] for i in range(m)], vex)
        g = cval(gotT[j])
        for p in range(2):
            assert abs(float(g[p] - want[p])) <= 2 * u * abs(float(want[p])) + 1e-300


def pin_matvec_conjT_gram(o):
    """Q^H q_j from the oracle's own MGS is a column of the identity up to O(kappa u)
    (Section 3); a transposed instead of conjugated product leaves O(1) cross terms."""
    A, _, _ = inputs.system(30, 12, 2, 6104)
    Q, R, st = o.qr(A.copy())
    assert st == 0
    for j in (0, 5, 11):
        col = o.matvec_conjT(Q, Q[j])
        e = np.zeros_like(col)
        e[j, 0, 0] = 1.0
        d, _ = o.max_abs_diff(col, e)
        assert d < 1e-28


def quick_battery(o):
    """Every pin at its smallest size; used on planted builds."""
    pin_error_free_transforms(o)
    for L in (2, 4):
        pin_real_ops(o, L, trials=40)
        pin_complex_ops(o, L, trials=20)
        pin_backsub(o, L)
        pin_mgs_special_cases(o, L)
        pin_mgs_exact_rational(o, L, cases=((3, 2), (4, 4)))
    pin_table2(o, "DD", 1, 3)
    pin_matvec(o, 2, 2)
    pin_matvec_conjT_gram(o)
