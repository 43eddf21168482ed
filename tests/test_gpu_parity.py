"""CUDA path vs the oracle, element by element (x, R, Q, z, residual), DD and QD.

Sizes span several row blocks and column groups, ragged row blocks and m > n."""

import numpy as np
import pytest

from helpers import TOL, compare_ls, gpu_qr, planted_system, rel, upper
from paper_1210_0800_gb300 import inputs

pytestmark = pytest.mark.gpu

DD_SHAPES = [(32, 32), (1, 1), (5, 1), (7, 3), (33, 33), (40, 24), (67, 45), (100, 100), (130, 97), (200, 64)]
QD_SHAPES = [(16, 16), (1, 1), (9, 4), (33, 20), (48, 48), (70, 33)]


@pytest.mark.parametrize("m,n", DD_SHAPES)
def test_ls_dd_vs_oracle(orc, m, n):
    A, xt, b = planted_system(m, n, 2, 7000 + m * 1000 + n, orc=orc)
    compare_ls(orc, A, b)


@pytest.mark.parametrize("m,n", QD_SHAPES)
def test_ls_qd_vs_oracle(orc, m, n):
    A, xt, b = planted_system(m, n, 4, 8000 + m * 1000 + n, orc=orc)
    compare_ls(orc, A, b)


@pytest.mark.parametrize("m,n,L", [(40, 24, 2), (64, 64, 2), (31, 17, 4)])
def test_ls_generic_rhs(orc, m, n, L):
    """Inconsistent right-hand side (nonzero residual z) as in a Newton step."""
    A, _, b = inputs.system(m, n, L, 9900 + m + n)
    errs, g, o = compare_ls(orc, A, b)
    if m > n:
        assert float(np.sum(o["z"])) > 0.1


@pytest.mark.parametrize("m,n,L", [(32, 32, 2), (50, 37, 2), (24, 24, 4)])
def test_qr_vs_oracle(orc, m, n, L):
    A = inputs.matrix_uniform(m, n, L, 5150 + m)
    Qg, Rg, st = gpu_qr(A.copy())
    Qo, Ro, sto = orc.qr(A.copy())
    assert st == 0 and sto == 0
    assert rel(orc, Qg, Qo) <= TOL[L]
    assert rel(orc, upper(Rg), upper(Ro)) <= TOL[L]


def test_status_rank_deficient(orc):
    A, _, b = inputs.system(20, 8, 2, 4321)
    A[3] = 0.0
    from helpers import gpu_ls_solve

    assert gpu_ls_solve(A, b)["status"] == 2


def test_status_nonfinite():
    A, _, b = inputs.system(20, 8, 2, 4322)
    A[2, 5, 0, 0] = np.nan
    from helpers import gpu_ls_solve

    assert gpu_ls_solve(A, b)["status"] == 3


def test_repeatable_bitwise(orc):
    """Two runs give bit-identical results (fixed reduction order)."""
    from helpers import gpu_ls_solve

    A, xt, b = planted_system(96, 80, 2, 1234, orc=orc)
    r1 = gpu_ls_solve(A.copy(), b.copy())
    r2 = gpu_ls_solve(A.copy(), b.copy())
    for k in ("x", "Q", "R", "z", "resid"):
        assert np.array_equal(r1[k], r2[k]), k
