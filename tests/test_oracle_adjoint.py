"""Pins of the oracle's least-squares adjoint (gradients of a real loss through
x = argmin ||b - A x||) against exact rational arithmetic and QD central differences."""

import math
from fractions import Fraction as F

import numpy as np
import pytest

import pins
from paper_1210_0800_gb300 import inputs


def exact_adjoint(Aex, bex, Gex):
    """w = (A^H A)^{-1} G, x = (A^H A)^{-1} A^H b, r = b - A x, grad_b = A w,
    grad_A = r w^H - grad_b x^H, all over the Gaussian rationals."""
    n, m = len(Aex), len(Aex[0])
    Gm = [[pins.cdot(Aex[i], Aex[j]) for j in range(n)] for i in range(n)]

    def solve(rhs):
        M = [row[:] + [rhs[i]] for i, row in enumerate(Gm)]
        for c in range(n):
            p = next(r for r in range(c, n) if M[r][c] != (0, 0))
            M[c], M[p] = M[p], M[c]
            for r in range(n):
                if r != c and M[r][c] != (0, 0):
                    f = pins.cdiv(M[r][c], M[c][c])
                    M[r] = [pins.csub(M[r][k], pins.cmul(f, M[c][k])) for k in range(n + 1)]
        return [pins.cdiv(M[i][n], M[i][i]) for i in range(n)]

    x = solve([pins.cdot(Aex[i], bex) for i in range(n)])
    w = solve(Gex)
    Aw = [pins.sum_cols(Aex, w, i) for i in range(m)]
    r = [pins.csub(bex[i], pins.sum_cols(Aex, x, i)) for i in range(m)]
    gA = [[pins.csub(pins.cmul(r[i], pins.cconj(w[j])), pins.cmul(Aw[i], pins.cconj(x[j]))) for i in range(m)]
          for j in range(n)]
    return gA, Aw, x


def adjoint_exact_pin(orc, L, m, n):
    """The oracle's gradients on Gaussian-integer systems against exact_adjoint."""
    u = 2.0 ** (-53 * L)
    for rep in range(2):
        seed = 700 + 10 * m + n + rep
        vals = pins.gaussian_int_matrix(m, n, seed)
        Aex = [[(F(vals[j, i, 0]), F(vals[j, i, 1])) for i in range(m)] for j in range(n)]
        if any(pins.cdot(v, v)[0] == 0 for v in pins.exact_cgs(Aex)):
            continue
        bv = inputs.uniform_int(seed + 1, 2 * m, -5, 5).astype(np.float64).reshape(m, 2)
        gv = inputs.uniform_int(seed + 2, 2 * n, -3, 3).astype(np.float64).reshape(n, 2)
        A, b, G = pins.embed(vals, L), pins.embed(bv, L), pins.embed(gv, L)
        gA, gb, x, st = orc.ls_adjoint(A, b, G)
        assert st == 0
        eA, eb, ex = exact_adjoint(Aex, [pins.cval(b[i]) for i in range(m)], [pins.cval(G[k]) for k in range(n)])
        scale = max(max(pins.cnorm_inf(v) for v in eb), max(pins.cnorm_inf(v) for col in eA for v in col), 1.0)
        tol = u * 2.0 ** 20 * scale
        for i in range(m):
            assert pins.cnorm_inf(pins.csub(pins.cval(gb[i]), eb[i])) <= tol, ("grad_b", i)
            for j in range(n):
                assert pins.cnorm_inf(pins.csub(pins.cval(gA[j, i]), eA[j][i])) <= tol, ("grad_A", i, j)


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("m,n", [(3, 3), (4, 4), (5, 3), (6, 4)])
def test_adjoint_exact_rational(orc, L, m, n):
    adjoint_exact_pin(orc, L, m, n)


def test_planted_adjoint_mistake_is_caught(tmp_path):
    """A build whose grad_A uses g x^T instead of g x^H fails the exact pin."""
    import oracle

    o = oracle.Oracle(oracle.build(plant=11, out=str(tmp_path / "liboracle_plant11.so")))
    assert o.plant() == 11
    with pytest.raises(AssertionError):
        adjoint_exact_pin(o, 2, 4, 4)


def loss(orc, A, b):
    """L = sum |x|^2 of the QD solve, exactly from the limbs."""
    r = orc.ls_solve(A.copy(), b.copy())
    return sum(pins.cabs2(pins.cval(r["x"][k])) for k in range(A.shape[0]))


def test_adjoint_matches_qd_finite_differences(orc):
    """Central differences with step 1e-20 of L = sum |x|^2 in quad-double match the
    gradient grad = dL/dRe + i dL/dIm for entries of A and b (G = 2x)."""
    m, n, L, h = 6, 4, 4, 1e-20
    A, _, b = inputs.system(m, n, L, 4711)
    x = orc.ls_solve(A.copy(), b.copy())["x"]
    G = 2.0 * x  # exact doubling of the limbs
    gA, gb, _, st = orc.ls_adjoint(A, b, G)
    assert st == 0
    hq = np.array([h, 0.0, 0.0, 0.0])

    def bump(arr, idx, part, sign):
        out = arr.copy()
        out[idx + (part,)] = orc.add(4, out[idx + (part,)], sign * hq)
        return out

    checks = [("A", (1, 2)), ("A", (3, 5)), ("A", (0, 0)), ("b", (4,)), ("b", (1,))]
    for which, idx in checks:
        for part in (0, 1):
            if which == "A":
                lp = loss(orc, bump(A, idx, part, 1.0), b)
                lm = loss(orc, bump(A, idx, part, -1.0), b)
                want = pins.fval(gA[idx][part])
            else:
                lp = loss(orc, A, bump(b, idx, part, 1.0))
                lm = loss(orc, A, bump(b, idx, part, -1.0))
                want = pins.fval(gb[idx][part])
            fd = (lp - lm) / (2 * F(h))
            assert abs(float(fd - want)) <= 1e-33 * max(1.0, abs(float(want))), (which, idx, part, float(fd), float(want))
