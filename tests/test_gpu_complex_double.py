"""Complex double variant (L = 1) against the oracle, and the paper's accuracy experiment
(Section 4, Table 2) reproduced with the GPU factorisations: log10 of Eq. 2's error of the
GPU's Q and R (evaluated exactly by the oracle) falls in the printed ranges."""

import math

import pytest

import pins
from helpers import compare_ls, gpu_qr, planted_system
from paper_1210_0800_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,n", [(32, 32), (7, 3), (67, 45), (130, 97)])
def test_ls_d_vs_oracle(orc, m, n):
    A, xt, b = planted_system(m, n, 1, 6100 + m + n, orc=orc)
    compare_ls(orc, A, b)


@pytest.mark.parametrize("prec,g,count", [("D", 1, 20), ("D", 8, 10), ("DD", 1, 20), ("DD", 16, 20)])
def test_table2_on_gpu(orc, prec, g, count):
    L = pins.PREC_L[prec]
    lo, hi = pins.load_table2()[(prec, g)]
    logs = []
    for s in range(count):
        A = inputs.complex_polar((32, 32), L, 777000 + s, g)
        Q, R, st = gpu_qr(A.copy())
        assert st == 0
        e, _ = orc.qr_error(A, Q, R)
        logs.append(math.log10(e))
    assert min(logs) >= lo - 0.5 and max(logs) <= hi + 0.5, (prec, g, min(logs), max(logs), lo, hi)


@pytest.mark.parametrize("g", [17, 32])
def test_table2_qd_on_gpu(orc, g):
    """Quad-double: the kernels' operations are faithful to about one unit of 2^-212 where
    the oracle's are exactly rounded (a few hundredths), and the update's rounding sets
    Eq. 2's error (tests/test_qd_error_sources.py); on the GB300 the GPU's log10 e lies 1.6
    to 2.1 decades above the oracle's on the same matrices (measured, g = 17 and 32), so it
    must stay within 2.5 decades of the oracle's and of the printed upper end, and far
    below double-double's."""
    lo, hi = pins.load_table2()[("QD", g)]
    for s in range(6):
        A = inputs.complex_polar((32, 32), 4, 777000 + s, g)
        Q, R, st = gpu_qr(A.copy())
        assert st == 0
        e = math.log10(orc.qr_error(A, Q, R)[0])
        Qo, Ro, _ = orc.qr(A.copy())
        eo = math.log10(orc.qr_error(A, Qo, Ro)[0])
        print("Table 2 QD g=%d matrix %d: log10 e GPU %.2f, oracle %.2f, printed [%.1f, %.1f]" % (g, s, e, eo, lo, hi))
        assert e <= eo + 2.5 and e <= hi + 2.5 and e >= lo - 0.5, (g, s, e, eo, lo, hi)
