"""The benchmarked workloads at their full sizes, in the launch configuration the
benchmark times (the default kernel for each size), checked against the oracle.

Where the oracle solves the system in seconds (m = n = 32 DD; m = n = 256 DD with
extreme scaling) the comparison is element by element; for m = 320, n = 256 QD the
oracle's solve takes minutes, so the result is checked through properties the oracle
computes exactly at this size: A = QR on sampled columns, Q^H Q = I on sampled columns
(Section 3), the optimality of x (A^H (b - A x) = 0, Eq. 1) and the residual column.
The ragged batch is sampled system by system."""

import math

import numpy as np
import pytest

from helpers import TOL, compare_ls, gpu_ls_solve, planted_system, rel, upper
from paper_1210_0800_gb300 import inputs

pytestmark = pytest.mark.gpu


def _amax(orc, X):
    return orc.max_abs_diff(X, 0 * X)[0]


def _kappa(orc, A, R):
    """kappa^ = ||A||_F ||R^-1||_F, R^-1 from the double-double leading limbs of R."""
    afro = math.sqrt(float(np.sum(A[..., 0] ** 2)))
    return afro * orc.rinv_fro(np.ascontiguousarray(R[..., :2]))


def test_c0_dd_32x32_vs_oracle(orc):
    A, _, b = inputs.system(32, 32, 2, inputs.system_seed(inputs.workload_seed("c0"), 0))
    compare_ls(orc, A, b)


def test_c2_dd_256_extreme_vs_oracle(orc):
    """Rows scaled by 10^U{-12..12}, columns by 10^U{-4..4}: x, R and Q against the
    oracle relative to kappa^ u (u = 2^-104), with the bound err <= 10 n kappa^ u."""
    m = n = 256
    A, _, b = inputs.system(m, n, 2, inputs.system_seed(inputs.workload_seed("c2"), 0), extreme=True)
    g = gpu_ls_solve(A.copy(), b.copy())
    o = orc.ls_solve(A.copy(), b.copy())
    assert g["status"] == 0 and o["status"] == 0
    kap = _kappa(orc, A, o["R"])
    u = 2.0 ** -104
    err = dict(x=rel(orc, g["x"], o["x"]), R=rel(orc, upper(g["R"]), upper(o["R"])), Q=rel(orc, g["Q"], o["Q"]))
    print("c2: kappa^ = %.3e, err/(kappa^ u) = %s" % (kap, {k: "%.3g" % (v / (kap * u)) for k, v in err.items()}))
    for k, v in err.items():
        assert v <= 10 * n * kap * u, (k, v, kap)


@pytest.mark.parametrize("m,n", [(64, 64), (90, 65), (160, 130)])
def test_qd_extreme_vs_oracle(orc, m, n):
    """The extreme scaling of the DD workload (rows 10^U{-12..12}, columns 10^U{-4..4}) in
    quad double, through the QD kernel's paired back substitution (n = 65: a block with an
    odd row count): x, R and Q against the oracle, err <= 10 n kappa^ u with u = 2^-209."""
    A, _, b = inputs.system(m, n, 4, 8800 + m + n, extreme=True)
    g = gpu_ls_solve(A.copy(), b.copy())
    o = orc.ls_solve(A.copy(), b.copy())
    assert g["status"] == 0 and o["status"] == 0
    kap = _kappa(orc, A, o["R"])
    u = 2.0 ** -209
    err = dict(x=rel(orc, g["x"], o["x"]), R=rel(orc, upper(g["R"]), upper(o["R"])), Q=rel(orc, g["Q"], o["Q"]))
    for k, v in err.items():
        assert v <= 10 * n * kap * u, (k, v, kap)


def test_c1_qd_320x256_properties(orc):
    m, n, L = 320, 256, 4
    u = 2.0 ** -209
    A, _, b = inputs.system(m, n, L, inputs.system_seed(inputs.workload_seed("c1"), 0))
    g = gpu_ls_solve(A.copy(), b.copy())
    assert g["status"] == 0
    Q, R, x = g["Q"], upper(g["R"]), g["x"]
    # R: real positive diagonal
    for j in range(n):
        assert R[j, j, 0, 0] > 0 and not R[j, j, 1].any()
    kap = _kappa(orc, A, R)
    amax = _amax(orc, A)
    # A = QR on sampled columns: backward error O(n u ||A||)
    for j in (0, 1, n // 2, n - 1):
        qr_j = orc.matvec(Q, R[j])
        d, _ = orc.max_abs_diff(qr_j, A[j])
        assert d <= 10 * n * u * amax, (j, d)
    # Q^H q_j = e_j on sampled columns: loss of orthogonality O(kappa u)
    for j in (0, n // 2, n - 1):
        col = orc.matvec_conjT(Q, Q[j])
        e = np.zeros_like(col)
        e[j, 0, 0] = 1.0
        d, _ = orc.max_abs_diff(col, e)
        assert d <= 10 * n * kap * u, (j, d, kap)
    # optimality of x: A^H r = 0 with r = b - A x computed exactly
    r, _ = orc.residual(A, b, x, Lout=L)
    ahr = orc.matvec_conjT(A, r)
    bound = 10 * n * kap * u * (m * amax * amax * _amax(orc, x) + amax * _amax(orc, b))
    assert _amax(orc, ahr) <= bound, (_amax(orc, ahr), bound)
    # what MGS leaves of b is the residual b - A x (Eq. 1) and z its norm
    d, _ = orc.max_abs_diff(g["resid"], r)
    assert d <= 10 * n * u * (m * amax * _amax(orc, x) + _amax(orc, b)), d
    rn = math.sqrt(sum(float(np.sum(r[i, :, 0] ** 2)) for i in range(m)))
    assert abs(float(np.sum(g["z"])) - rn) <= 1e-12 * rn


def test_c1_qd_planted_solution(orc):
    """b = A x_true at the same size: x recovers x_true to O(n kappa u)."""
    m, n, L = 320, 256, 4
    A, xt, b = planted_system(m, n, L, inputs.system_seed(inputs.workload_seed("c1"), 1), orc=orc)
    g = gpu_ls_solve(A.copy(), b.copy())
    assert g["status"] == 0
    kap = _kappa(orc, A, upper(g["R"]))
    assert rel(orc, g["x"], xt) <= 10 * n * kap * 2.0 ** -209


def test_c3_batched_512_sampled(orc):
    """The 512-system ragged DD batch, as benchmarked: every status clean, eight systems
    (the largest, the smallest and six more) against the oracle."""
    import torch

    import paper_1210_0800_gb300 as mg

    systems = inputs.ragged_batch(2, 512, (16, 192), (0, 16), inputs.system_seed(inputs.workload_seed("c3"), 0))
    bt = mg.make_batch(systems, torch.device("cuda:0"), largest_first=True)
    st = mg.ls_solve_batched(bt).cpu().numpy()
    torch.cuda.synchronize()
    assert (st == 0).all()
    sizes = [A.shape[0] * A.shape[1] for A, _ in systems]
    pick = {int(np.argmax(sizes)), int(np.argmin(sizes))} | set(range(5, 512, 85))
    for i in sorted(pick):
        A, b = systems[i]
        n, m = A.shape[0], A.shape[1]
        xo = int(bt.x_off[i])
        x = bt.x_pool[xo:xo + n].cpu().numpy()
        o = orc.ls_solve(A.copy(), b.copy())
        assert rel(orc, x, o["x"]) <= TOL[2], i
