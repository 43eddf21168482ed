"""Degenerate cases of the method with exactly known results, and the largest systems a
single solve supports (the next size up is refused on the host)."""

import numpy as np
import pytest

from helpers import gpu_ls_solve, gpu_qr, planted_system, upper
from paper_1210_0800_gb300 import inputs

pytestmark = pytest.mark.gpu


def _amax(orc, X):
    return orc.max_abs_diff(X, 0 * X)[0]


@pytest.mark.parametrize("L", [1, 2, 4])
def test_zero_rhs(L):
    """b = 0: y = Q^H b = 0, so x = 0, the residual column stays 0 and z = 0 (Eq. 1)."""
    A, _, b = inputs.system(70, 50, L, 9101)
    g = gpu_ls_solve(A, np.zeros_like(b))
    assert g["status"] == 0
    assert not g["x"].any() and not g["resid"].any() and not g["z"].any()


@pytest.mark.parametrize("L", [2, 4])
def test_rhs_orthogonal_to_range(orc, L):
    """Columns of A along the first n unit vectors (complex multiples), b in the span of
    the others: every projection r_kj of b is exactly 0, so x = 0, the residual is b and
    z = ||b|| (Section 3, Eq. 1)."""
    m, n = 40, 24
    A = np.zeros((n, m, 2, L))
    d = inputs.complex_uniform((n,), L, 9102)
    for j in range(n):
        A[j, j] = d[j]
    b = np.zeros((m, 2, L))
    b[n:] = inputs.complex_uniform((m - n,), L, 9103)
    g = gpu_ls_solve(A.copy(), b.copy())
    assert g["status"] == 0
    assert not g["x"].any()
    assert orc.max_abs_diff(g["resid"], b)[0] == 0.0
    want = np.sqrt(np.sum(b[n:, :, 0] ** 2))
    assert abs(float(np.sum(g["z"])) - want) <= 1e-15 * want


@pytest.mark.parametrize("L", [2, 4])
def test_upper_triangular_is_its_own_r(L):
    """A upper triangular with powers of two on the diagonal and small integers above it
    (m = n): every projection c_kj = G_kj / G_kk, square root and update is exact, so
    Q = I and R = A exactly (Figure 1)."""
    n = 20
    A = np.zeros((n, n, 2, L))
    vals = inputs.uniform_int(9104, n * n * 2, -9, 9).reshape(n, n, 2)
    for j in range(n):
        for i in range(j):
            A[j, i, :, 0] = vals[j, i]
        A[j, j, 0, 0] = 2.0 ** (abs(int(vals[j, j, 0])) % 4)
    Q, R, st = gpu_qr(A.copy())
    assert st == 0
    eye = np.zeros_like(Q)
    for j in range(n):
        eye[j, j, 0, 0] = 1.0
    assert np.array_equal(Q, eye)
    assert np.array_equal(upper(R), A)


@pytest.mark.parametrize("L", [2, 4])
def test_orthogonal_columns_give_diagonal_r(orc, L):
    """Columns of a Fourier matrix are orthogonal with norm sqrt(m): R is sqrt(m) I up to
    rounding (the off-diagonal projections cancel to the working precision)."""
    m = n = 16
    A = np.zeros((n, m, 2, L))
    for j in range(n):
        for i in range(m):
            ang = 2 * np.pi * ((i * j) % m) / m
            A[j, i, 0, 0] = np.cos(ang)
            A[j, i, 1, 0] = np.sin(ang)
    Q, R, st = gpu_qr(A.copy())
    assert st == 0
    Ru = upper(R)
    u = 2.0 ** (-53 * L)
    for j in range(n):
        assert abs(Ru[j, j, 0, 0] - 4.0) <= 1e-14  # the double values of cos/sin are not exact
        off = Ru[j, :j]
        assert np.abs(off[..., 0]).max(initial=0.0) <= 1e-14
    # orthogonality of the computed Q to the working precision
    for j in (0, 7, 15):
        col = orc.matvec_conjT(Q, Q[j])
        e = np.zeros_like(col)
        e[j, 0, 0] = 1.0
        assert orc.max_abs_diff(col, e)[0] <= 100 * n * u


def _largest_square(L):
    import paper_1210_0800_gb300 as mg

    lo, hi = 64, 8192
    assert mg.mgs_workspace_bytes(L, lo, lo, True) > 0
    while mg.mgs_workspace_bytes(L, hi, hi, True) > 0:
        hi *= 2
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if mg.mgs_workspace_bytes(L, mid, mid, True) > 0:
            lo = mid
        else:
            hi = mid
    return lo


@pytest.mark.parametrize("L", [2, 4])
def test_largest_supported_square_system(orc, L):
    """The largest m = n one solve holds: it runs clean and its x is backward stable
    (||b - A x|| = O(n u ||A|| ||x||), exact residual); one size up is refused with
    MGS_ENOSPACE before any launch."""
    import torch

    import paper_1210_0800_gb300 as mg

    n = _largest_square(L)
    assert n >= 512
    print("largest square system, limbs %d: n = %d" % (L, n))
    A, xt, b = planted_system(n, n, L, 9200 + L, orc=orc)
    g = gpu_ls_solve(A.copy(), b.copy(), with_R=False)
    assert g["status"] == 0
    _, nrm2 = orc.residual(A, b, g["x"], Lout=L)
    u = 2.0 ** (-53 * L)
    assert np.sqrt(nrm2) <= 10 * n * u * n * _amax(orc, A) * _amax(orc, g["x"])
    At = torch.zeros((n + 1, n + 1, 2, L), dtype=torch.float64, device="cuda:0")
    bt = torch.zeros((n + 1, 2, L), dtype=torch.float64, device="cuda:0")
    with pytest.raises(mg.MGSError) as ei:
        {2: mg.ls_solve_dd, 4: mg.ls_solve_qd}[L](At, bt)
    assert ei.value.code == 6
