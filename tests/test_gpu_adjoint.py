"""Differentiated least squares: the GPU adjoint against the oracle adjoint (itself
pinned by exact rationals and QD finite differences), through torch.autograd, with and
without recomputation of the factors; a full-size system against the oracle; and the DD
gradient against QD central differences of the GPU quad-double solve on sampled entries."""

import numpy as np
import pytest
import torch

from helpers import rel
from paper_1210_0800_gb300 import inputs

pytestmark = pytest.mark.gpu


def uniform(orc, B, m, n, L, seed):
    As, bs = [], []
    for i in range(B):
        A, _, b = inputs.system(m, n, L, inputs.system_seed(seed, i))
        As.append(A)
        bs.append(b)
    return np.stack(As), np.stack(bs)


def grads_gpu(A, b, budget=None):
    import paper_1210_0800_gb300 as mg

    dev = torch.device("cuda:0")
    At = torch.from_numpy(A).to(dev).requires_grad_(True)
    bt = torch.from_numpy(b).to(dev).requires_grad_(True)
    kw = {} if budget is None else {"save_budget": budget}
    x = mg.lstsq(At, bt, **kw)
    x.backward(gradient=2.0 * x.detach())  # L = sum |x|^2  ->  dL/dx = 2x (exact on limbs)
    torch.cuda.synchronize()
    return x.detach().cpu().numpy(), At.grad.cpu().numpy(), bt.grad.cpu().numpy()


@pytest.mark.parametrize("B,m,n", [(3, 20, 12), (2, 41, 33)])
def test_adjoint_vs_oracle(orc, B, m, n):
    A, b = uniform(orc, B, m, n, 2, 7700 + m)
    x, gA, gb = grads_gpu(A, b)
    for i in range(B):
        ox = orc.ls_solve(A[i].copy(), b[i].copy())["x"]
        oA, ob, _, st = orc.ls_adjoint(A[i], b[i], 2.0 * ox)
        assert st == 0
        assert rel(orc, x[i], ox) <= 1e-26
        assert rel(orc, gA[i], oA) <= 1e-25, i
        assert rel(orc, gb[i], ob) <= 1e-25, i


def test_recompute_path_is_identical(orc):
    """Recomputing Q, R in the backward gives the same gradients as saving them."""
    A, b = uniform(orc, 3, 24, 16, 2, 7800)
    _, gA0, gb0 = grads_gpu(A, b)
    _, gA1, gb1 = grads_gpu(A, b, budget=0)
    assert np.array_equal(gA0, gA1) and np.array_equal(gb0, gb1)


def test_full_size_system_vs_oracle(orc):
    """m=160, n=128 (the differentiated workload's shape), one system against the oracle."""
    A, b = uniform(orc, 1, 160, 128, 2, 7900)
    x, gA, gb = grads_gpu(A, b)
    ox = orc.ls_solve(A[0].copy(), b[0].copy())["x"]
    oA, ob, _, _ = orc.ls_adjoint(A[0], b[0], 2.0 * ox)
    assert rel(orc, gA[0], oA) <= 1e-24
    assert rel(orc, gb[0], ob) <= 1e-24


def test_dd_gradient_vs_qd_central_differences(orc):
    """Consistency of the DD adjoint with QD central differences (step 1e-20) of the GPU
    quad-double solve, on 8 random entries of A and b per system."""
    import paper_1210_0800_gb300 as mg

    B, m, n, h = 2, 40, 32, 1e-20
    A, b = uniform(orc, B, m, n, 2, 8000)
    _, gA, gb = grads_gpu(A, b)
    dev = torch.device("cuda:0")

    from fractions import Fraction as F

    def solve_qd(Aq, bq):
        x, st = mg.ls_solve_qd(torch.from_numpy(Aq).to(dev), torch.from_numpy(bq).to(dev))
        assert int(st.item()) == 0
        return x.cpu().numpy()

    def L_of(xs):
        s = F(0)
        for k in range(xs.shape[0]):
            re = sum(F(float(v)) for v in xs[k, 0])
            im = sum(F(float(v)) for v in xs[k, 1])
            s += re * re + im * im
        return s

    rng = inputs.uniform_int(8001, 64, 0, 10 ** 6)
    for i in range(B):
        A4 = np.zeros((n, m, 2, 4))
        A4[..., :2] = A[i]
        b4 = np.zeros((m, 2, 4))
        b4[..., :2] = b[i]
        for t in range(8):
            which = "A" if t < 6 else "b"
            part = int(rng[8 * i + t] % 2)
            if which == "A":
                jj, ii = int(rng[8 * i + t] // 2 % n), int(rng[8 * i + t] // 7 % m)
                Ap, Am = A4.copy(), A4.copy()
                Ap[jj, ii, part] = orc.add(4, Ap[jj, ii, part], np.array([h, 0, 0, 0]))
                Am[jj, ii, part] = orc.add(4, Am[jj, ii, part], np.array([-h, 0, 0, 0]))
                fd = (L_of(solve_qd(Ap, b4)) - L_of(solve_qd(Am, b4))) / (2 * F(h))
                want = sum(F(float(v)) for v in gA[i][jj, ii, part])
            else:
                ii = int(rng[8 * i + t] // 3 % m)
                bp, bm = b4.copy(), b4.copy()
                bp[ii, part] = orc.add(4, bp[ii, part], np.array([h, 0, 0, 0]))
                bm[ii, part] = orc.add(4, bm[ii, part], np.array([-h, 0, 0, 0]))
                fd = (L_of(solve_qd(A4, bp)) - L_of(solve_qd(A4, bm))) / (2 * F(h))
                want = sum(F(float(v)) for v in gb[i][ii, part])
            assert abs(float(fd - want)) <= 1e-26 * max(1.0, abs(float(want))), (i, which, float(fd), float(want))


@pytest.mark.parametrize("B,m,n", [(2, 18, 12), (2, 30, 24)])
def test_qd_adjoint_vs_oracle(orc, B, m, n):
    """The quad-double adjoint (ls_adjoint_qd_batched through lstsq) against the oracle."""
    A, b = uniform(orc, B, m, n, 4, 7950 + m)
    x, gA, gb = grads_gpu(A, b)
    for i in range(B):
        ox = orc.ls_solve(A[i].copy(), b[i].copy())["x"]
        oA, ob, _, st = orc.ls_adjoint(A[i], b[i], 2.0 * ox)
        assert st == 0
        assert rel(orc, x[i], ox) <= 1e-56
        assert rel(orc, gA[i], oA) <= 1e-55, i
        assert rel(orc, gb[i], ob) <= 1e-55, i


def test_complex_double_is_refused():
    import torch

    import paper_1210_0800_gb300 as mg

    A = torch.zeros((1, 3, 4, 2, 1), dtype=torch.float64, device="cuda:0")
    b = torch.zeros((1, 4, 2, 1), dtype=torch.float64, device="cuda:0")
    with pytest.raises(ValueError):
        mg.lstsq(A, b)
