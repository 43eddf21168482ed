"""Pins of the oracle's Gram-Schmidt least squares (Figure 1, Eq. 1, Figure 3, Table 2)."""

import math

import numpy as np
import pytest

import pins
from paper_1210_0800_gb300 import inputs


@pytest.mark.parametrize("L", [2, 4])
def test_exact_rational(orc, L):
    pins.pin_mgs_exact_rational(orc, L)


@pytest.mark.parametrize("L", [1, 2, 4])
def test_special_cases(orc, L):
    pins.pin_mgs_special_cases(orc, L)


@pytest.mark.parametrize("L", [1, 2, 4])
def test_backsub(orc, L):
    pins.pin_backsub(orc, L)


@pytest.mark.parametrize(
    "prec,g,count",
    [("D", 1, 40), ("D", 8, 20), ("DD", 1, 40), ("DD", 8, 20), ("DD", 16, 30), ("QD", 17, 8), ("QD", 32, 8)],
)
def test_table2(orc, prec, g, count):
    pins.pin_table2(orc, prec, g, count)


def test_table2_precision_ordering(orc):
    """Each extra limb pair buys ~16 decimal digits at the same g (Table 2's D/DD columns
    are 16 decades apart; DD/QD 32 decades at g=17 and 32)."""
    d = np.mean(pins.table2_logs(orc, "D", 1, 10))
    dd = np.mean(pins.table2_logs(orc, "DD", 1, 10))
    assert 14.5 < d - dd < 17.5


@pytest.mark.parametrize("L,m,n", [(2, 48, 40), (4, 24, 20), (2, 33, 33)])
def test_invariants(orc, L, m, n):
    """Q^H Q = I and A = QR up to O(kappa u) and O(n u); z equals ||b - A x|| (Eq. 1);
    the reduced last column equals b - A x; a planted x_true is recovered."""
    u = 2.0 ** (-53 * L)
    A, xt, _ = inputs.system(m, n, L, 9100 + m)
    b = orc.matvec(A, xt)
    res = orc.ls_solve(A, b)
    assert res["status"] == 0
    rinv = orc.rinv_fro(res["R"])
    afro = math.sqrt(float(np.sum(A[..., 0] ** 2)))
    kappa = afro * rinv
    orth = orc.orth_error(res["Q"])
    assert orth <= 50 * kappa * u
    e, _ = orc.qr_error(A, res["Q"], res["R"])
    amax = float(np.max(np.abs(A[..., 0])))
    assert e <= 10 * n * u * amax * math.sqrt(m)
    # planted solution
    d, xm = orc.max_abs_diff(res["x"], xt)
    assert d / xm <= 10 * kappa * u * n
    # residual identity: z = ||b - A x||, and the reduced last column is b - A x
    r, nrm2 = orc.residual(A, b, res["x"], Lout=L)
    z = float(sum(res["z"]))
    bnorm = math.sqrt(float(np.sum(b[..., 0] ** 2)))
    assert abs(z - math.sqrt(max(nrm2, 0.0))) <= 10 * kappa * u * bnorm
    dres, _ = orc.max_abs_diff(res["resid"], r)
    assert dres <= 10 * kappa * u * bnorm


def test_inconsistent_residual_identity(orc):
    """Generic b (m > n): ||b - A x||^2 = z^2 (Eq. 1 with R x = y exactly), and the
    residual is orthogonal to the columns of A."""
    L, m, n = 2, 40, 24
    u = 2.0 ** -106
    A, _, b = inputs.system(m, n, L, 9300)
    res = orc.ls_solve(A, b)
    _, nrm2 = orc.residual(A, b, res["x"], Lout=L)
    z = float(sum(res["z"]))
    assert z > 0.5  # generic b is far from the range of A
    assert abs(z * z - nrm2) <= 1e4 * u * nrm2
    # A^H r = 0 (normal equations) up to rounding
    Ah = A[..., 0, 0] - 1j * A[..., 1, 0]
    rr = res["resid"][:, 0, 0] + 1j * res["resid"][:, 1, 0]
    assert np.max(np.abs(Ah @ rr)) <= 1e-13 * math.sqrt(nrm2) * math.sqrt(m)


def test_rank_deficient_status(orc):
    """No pivoting (Section 4): a zero column gives the rank-deficiency status 2."""
    A, _, b = inputs.system(8, 4, 2, 9400)
    A[2] = 0.0
    assert orc.ls_solve(A, b)["status"] == 2
    Q, R, st = orc.qr(A)
    assert st == 2


def test_dd_qd_agree(orc):
    """The same DD-representable system solved at L=2 and L=4 agrees to DD accuracy."""
    A2, xt2, _ = inputs.system(20, 16, 2, 9500)
    A4 = np.zeros(A2.shape[:-1] + (4,))
    A4[..., :2] = A2
    x4 = np.zeros(xt2.shape[:-1] + (4,))
    x4[..., :2] = xt2
    b4 = orc.matvec(A4, x4, Lout=4)
    b2 = orc.matvec(A2, xt2, Lout=2)
    r2 = orc.ls_solve(A2, b2)
    r4 = orc.ls_solve(A4, b4)
    d, xm = orc.max_abs_diff(r2["x"], r4["x"])
    assert d / xm < 1e-27


@pytest.mark.parametrize("L,Lout", [(1, 2), (2, 2), (2, 4), (4, 4)])
def test_matvec_exact(orc, L, Lout):
    """A x and A^H v against exact rational arithmetic: every entry within one rounding to
    Lout limbs of the exact sum (the sums have cancellation: v = A x for some rows)."""
    m, n = 7, 5
    A = inputs.matrix_uniform(m, n, L, 6101)
    x = inputs.system(m, n, L, 6102)[1]
    v = inputs.system(m, n, L, 6103)[2]
    v[3] = orc.matvec(A, x)[3]  # a row that is itself a combination of the columns
    Aex = [[pins.cval(A[j, i]) for j in range(n)] for i in range(m)]
    xex = [pins.cval(x[j]) for j in range(n)]
    vex = [pins.cval(v[i]) for i in range(m)]
    got = orc.matvec(A, x, Lout=Lout)
    gotT = orc.matvec_conjT(A, v, Lout=Lout)
    u = 2.0 ** (-53 * Lout)
    for i in range(m):
        want = (sum((pins.cmul(Aex[i][j], xex[j])[0] for j in range(n)), pins.F(0)),
                sum((pins.cmul(Aex[i][j], xex[j])[1] for j in range(n)), pins.F(0)))
        g = pins.cval(got[i])
        for p in range(2):
            assert abs(float(g[p] - want[p])) <= 2 * u * abs(float(want[p])) + 1e-300
    for j in range(n):
        want = pins.cdot([Aex[i][j] for i in range(m)], vex)
        g = pins.cval(gotT[j])
        for p in range(2):
            assert abs(float(g[p] - want[p])) <= 2 * u * abs(float(want[p])) + 1e-300


def test_matvec_conjT_gram(orc):
    """Q^H q_j from the oracle's own MGS is a column of the identity up to O(kappa u)
    (Section 3); a planted transposition (A^T instead of A^H) would leave the imaginary
    cross terms at O(1)."""
    A, _, _ = inputs.system(30, 12, 2, 6104)
    Q, R, st = orc.qr(A.copy())
    assert st == 0
    for j in (0, 5, 11):
        col = orc.matvec_conjT(Q, Q[j])
        e = np.zeros_like(col)
        e[j, 0, 0] = 1.0
        d, _ = orc.max_abs_diff(col, e)
        assert d < 1e-28


@pytest.mark.parametrize("L", [2, 4])
def test_newton_linear_one_step(orc, L):
    """For F(x) = A x - b the Newton step from any x0 lands on the least-squares solution:
    x0 - argmin ||(A x0 - b) - A s|| = argmin ||b - A x|| (Section 7 with a linear system)."""
    A, x0, b = inputs.system(14, 9, L, 6201)
    ax = orc.matvec(A, x0, Lout=L)
    F = np.empty_like(ax)
    for i in range(14):
        for p in range(2):
            F[i, p] = orc.sub(L, ax[i, p], b[i, p])
    x1, s, z, st = orc.newton_step(A.copy(), F, x0)
    ref = orc.ls_solve(A.copy(), b.copy())
    assert st == 0
    d, xm = orc.max_abs_diff(x1, ref["x"])
    assert d / xm < (1e-27 if L == 2 else 1e-58)


def test_newton_quadratic_convergence(orc):
    """On a quadratic system with a planted root the oracle's Newton iterates converge
    quadratically (e_{k+1} <= C e_k^2) down to rounding level."""
    import newton_problem as npb

    m, n, L = 12, 8, 2
    A, c, b, xs = npb.problem(orc, m, n, L, 6202)
    x = xs.copy()
    x[..., 0] += 1e-3 * inputs.uniform_pm1(6203, x[..., 0].size).reshape(x[..., 0].shape)
    errs = []
    for _ in range(6):
        J, F = npb.evaluate(orc, A, c, b, x)
        x, s, z, st = orc.newton_step(J, F, x)
        assert st == 0
        errs.append(orc.max_abs_diff(x, xs)[0])
    assert errs[-1] < 1e-28
    for e0, e1 in zip(errs, errs[1:]):
        if e0 > 1e-14:
            assert e1 <= 50 * e0 * e0, errs
