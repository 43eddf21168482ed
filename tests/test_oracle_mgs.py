"""Pins of the oracle's Gram-Schmidt least squares (Figure 1, Eq. 1, Figure 3, Table 2)."""

import math

import numpy as np
import pytest

import pins
from paper_1210_0800_gb300 import inputs


@pytest.mark.parametrize("L", [2, 4, 8])
def test_exact_rational(orc, L):
    pins.pin_mgs_exact_rational(orc, L)


@pytest.mark.parametrize("L", [1, 2, 4, 8])
def test_special_cases(orc, L):
    pins.pin_mgs_special_cases(orc, L)


@pytest.mark.parametrize("L", [1, 2, 4, 8])
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
    pins.pin_matvec(orc, L, Lout)


def test_matvec_conjT_gram(orc):
    pins.pin_matvec_conjT_gram(orc)


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
