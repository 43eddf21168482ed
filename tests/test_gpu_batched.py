"""Batched ragged solve vs the oracle, system by system (x, Q, residual), DD and QD;
per-system statuses; independence of the hand-out order and of the launch shape."""

import numpy as np
import pytest

from helpers import TOL, rel
from paper_1210_0800_gb300 import inputs

pytestmark = pytest.mark.gpu


def ragged(orc, L, count, seed, n_lo=1, n_hi=40, extra_hi=8):
    ms, ns = inputs.ragged_shapes(count, seed, n_lo, n_hi, 0, extra_hi)
    systems = []
    for i, (m, n) in enumerate(zip(ms, ns)):
        A, xt, _ = inputs.system(int(m), int(n), L, inputs.system_seed(seed, i))
        systems.append((A, orc.matvec(A, xt)))
    return systems


def run(systems, tune=None, largest_first=True, order=None):
    import torch

    import paper_1210_0800_gb300 as mg

    bt = mg.make_batch(systems, torch.device("cuda:0"), largest_first=largest_first, order=order)
    st = mg.ls_solve_batched(bt, tune=tune)
    torch.cuda.synchronize()
    return bt, st.cpu().numpy()


def unpack(bt, i, systems):
    A, b = systems[i]
    n, m = A.shape[0], A.shape[1]
    ao, bo, xo = int(bt.a_off[i]), int(bt.b_off[i]), int(bt.x_off[i])
    Q = bt.A_pool[ao:ao + m * n].cpu().numpy().reshape(A.shape)
    r = bt.b_pool[bo:bo + m].cpu().numpy()
    x = bt.x_pool[xo:xo + n].cpu().numpy()
    return Q, r, x


@pytest.mark.parametrize("L,count,seed", [(2, 48, 61), (4, 16, 62)])
def test_batched_vs_oracle(orc, L, count, seed):
    systems = ragged(orc, L, count, seed)
    bt, st = run(systems)
    assert (st == 0).all(), st
    for i, (A, b) in enumerate(systems):
        Q, r, x = unpack(bt, i, systems)
        o = orc.ls_solve(A.copy(), b.copy())
        assert rel(orc, x, o["x"]) <= TOL[L], i
        assert rel(orc, Q, o["Q"]) <= TOL[L], i
        d, _ = orc.max_abs_diff(r, o["resid"])
        assert d <= TOL[L] * max(1.0, orc.max_abs_diff(b, 0 * b)[0]), i


def test_batched_shapes_and_order_agree(orc):
    """Every launch shape, chunk cap and hand-out order solves the batch to the same
    tolerance."""
    systems = ragged(orc, 2, 24, 63)
    ref, _ = run(systems, tune=None, largest_first=False)
    for tune, order in [((128, 1), "largest"), ((256, 1), "largest"), ((128, 3), "largest"), ((256, 2), "largest"),
                        ((256, 1, 0, 4), "largest"), ((128, 2, 0, 8), "interleave"), ((256, 1, 2, 16), "interleave"),
                        ((256, 1, 1, 1), "natural")]:
        bt, st = run(systems, tune=tune, order=order)
        assert (st == 0).all()
        for i in range(len(systems)):
            x0 = unpack(ref, i, systems)[2]
            x1 = unpack(bt, i, systems)[2]
            assert rel(orc, x1, x0) <= 1e-26, (tune, order, i)


def test_batched_statuses(orc):
    """A rank-deficient system reports MGS_ERANK and a non-finite one MGS_ENONFINITE;
    the others are unaffected."""
    systems = ragged(orc, 2, 6, 64)
    A, b = systems[2]
    A = A.copy()
    A[0] = 0.0
    systems[2] = (A, b)
    A4, b4 = systems[4]
    b4 = b4.copy()
    b4[0, 0, 0] = np.inf
    systems[4] = (A4, b4)
    bt, st = run(systems)
    assert st[2] == 2 and st[4] == 3
    for i in (0, 1, 3, 5):
        assert st[i] == 0
        o = orc.ls_solve(systems[i][0].copy(), systems[i][1].copy())
        assert rel(orc, unpack(bt, i, systems)[2], o["x"]) <= TOL[2]


def test_autotuner_searches_and_agrees_with_oracle(orc, tmp_path):
    """The tuner times shapes, splits, chunk caps and hand-out orders, caches its choice per
    shape bucket, and the tuned launch agrees with the oracle on a sample of the batch."""
    import torch

    import paper_1210_0800_gb300 as mg
    from paper_1210_0800_gb300 import tune

    systems = ragged(orc, 2, 40, 65, 8, 40)
    bt = mg.make_batch(systems, torch.device("cuda:0"))
    best, order, times = tune.tune_batched(bt, reps=1, cache_path=str(tmp_path / "c.json"))
    assert order in tune.ORDERS
    labels = set(times)
    assert any(lb.split(",")[4] == "interleave" for lb in labels)
    assert {int(lb.split(",")[2]) for lb in labels} >= set(tune.SPLITS)
    assert {int(lb.split(",")[3]) for lb in labels} >= {c for c in tune.CHUNKS if c <= best[0]}
    assert tune._label(tuple(best), order) in times
    again, order2, _ = tune.tune_batched(bt, cache_path=str(tmp_path / "c.json"))
    assert tuple(again) == tuple(best) and order2 == order
    bt2, st = run(systems, tune=tuple(best), order=order)
    assert (st == 0).all()
    for i in range(0, len(systems), 5):
        A, b = systems[i]
        x = unpack(bt2, i, systems)[2]
        assert rel(orc, x, orc.ls_solve(A.copy(), b.copy())["x"]) <= TOL[2], i


@pytest.mark.parametrize("L,split", [(2, 2), (2, 4), (4, 2), (1, 4)])
def test_split_systems_vs_oracle(orc, L, split):
    """Systems shared by a cluster of 2 or 4 CTAs (row slices, partials summed through
    distributed shared memory) agree with the oracle; tiny systems leave slices empty."""
    systems = ragged(orc, L, 12, 64 + split + L, n_lo=1, n_hi=60, extra_hi=12)
    bt, st = run(systems, tune=(256, 1, split))
    assert (st == 0).all(), st
    for i, (A, b) in enumerate(systems):
        Q, r, x = unpack(bt, i, systems)
        o = orc.ls_solve(A.copy(), b.copy())
        assert rel(orc, x, o["x"]) <= TOL[L], i
        assert rel(orc, Q, o["Q"]) <= TOL[L], i
        d, _ = orc.max_abs_diff(r, o["resid"])
        assert d <= TOL[L] * max(1.0, orc.max_abs_diff(b, 0 * b)[0]), i


def test_split_statuses(orc):
    """Per-system statuses with split systems: a rank-deficient and a non-finite system
    among clean ones, the non-finite entry in a slice other than rank 0's."""
    systems = ragged(orc, 2, 6, 65, n_lo=8, n_hi=20, extra_hi=40)
    A, b = systems[1]
    A[2] = 0.0
    A, b = systems[3]
    A[1, A.shape[1] - 1, 0, 0] = np.inf
    bt, st = run(systems, tune=(128, 1, 4))
    assert st[1] == 2 and st[3] == 3
    assert (np.delete(st, [1, 3]) == 0).all(), st


def test_automatic_split_for_small_batches(orc):
    """A batch much smaller than the GPU is split automatically and still agrees."""
    import torch

    import paper_1210_0800_gb300 as mg

    systems = ragged(orc, 2, 16, 66, n_lo=60, n_hi=90, extra_hi=16)
    bt, st = run(systems)
    assert (st == 0).all()
    for i in (0, 7, 15):
        A, b = systems[i]
        Q, r, x = unpack(bt, i, systems)
        assert rel(orc, x, orc.ls_solve(A.copy(), b.copy())["x"]) <= TOL[2]


@pytest.mark.parametrize("L,split", [(2, 1), (2, 2), (4, 1), (1, 4)])
def test_batched_packed_r_vs_oracle(orc, L, split):
    """The optional packed R of the batched solve (element (k, j), k <= j, at j(j+1)/2 + k;
    the forward output the adjoint reuses) agrees with the oracle's R, system by system,
    in one CTA per system and split over a cluster."""
    import torch

    import paper_1210_0800_gb300 as mg

    systems = ragged(orc, L, 10, 67 + L + split, n_lo=1, n_hi=48, extra_hi=10)
    bt = mg.make_batch(systems, torch.device("cuda:0")).with_R()
    st = mg.ls_solve_batched(bt, tune=(256, 1, split)).cpu().numpy()
    torch.cuda.synchronize()
    assert (st == 0).all()
    for i, (A, b) in enumerate(systems):
        n = A.shape[0]
        o = orc.ls_solve(A.copy(), b.copy())
        ro = int(bt.r_off[i])
        packed = bt.R_pool[ro:ro + n * (n + 1) // 2].cpu().numpy()
        R = np.zeros_like(o["R"])
        for j in range(n):
            R[j, :j + 1] = packed[j * (j + 1) // 2:j * (j + 1) // 2 + j + 1]
        Ro = o["R"].copy()
        for j in range(n):
            Ro[j, j + 1:] = 0.0
        assert rel(orc, R, Ro) <= TOL[L], i
