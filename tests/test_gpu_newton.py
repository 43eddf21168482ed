"""Newton corrector on the device (newton_step_*) against the oracle's Newton iteration on
the same nonlinear system; the device-side gate (converged or failed runs do nothing);
a run captured in a CUDA graph."""

import numpy as np
import pytest

import newton_problem as npb
from helpers import rel
from paper_1210_0800_gb300 import inputs

pytestmark = pytest.mark.gpu


def _start(xs, seed, eps=1e-3):
    x = xs.copy()
    x[..., 0] += eps * inputs.uniform_pm1(seed, x[..., 0].size).reshape(x[..., 0].shape)
    return x


def _oracle_run(orc, A, c, b, x, steps):
    xs = []
    for _ in range(steps):
        J, F = npb.evaluate(orc, A, c, b, x)
        x, _, _, st = orc.newton_step(J, F, x)
        assert st == 0
        xs.append(x.copy())
    return xs


@pytest.mark.parametrize("m,n,L", [(40, 32, 2), (20, 16, 4), (33, 33, 2), (24, 18, 1)])
def test_newton_vs_oracle(orc, m, n, L):
    import torch

    import paper_1210_0800_gb300 as mg

    A, c, b, xs = npb.problem(orc, m, n, L, 7300 + m + L)
    x0 = _start(xs, 7301)
    steps = 7 if L == 4 else 6  # quadratic convergence from 1e-3 to the rounding level
    want = _oracle_run(orc, A, c, b, x0.copy(), steps)
    dev = torch.device("cuda:0")
    x = torch.from_numpy(x0.copy()).to(dev)
    got = []

    def evaluate(xd, J, F):
        Jh, Fh = npb.evaluate(orc, A, c, b, xd.cpu().numpy())
        J.copy_(torch.from_numpy(Jh))
        F.copy_(torch.from_numpy(Fh))

    state = mg.NewtonState(dev)
    J = torch.empty(A.shape, dtype=torch.float64, device=dev)
    F = torch.empty(b.shape, dtype=torch.float64, device=dev)
    ws = st = None
    for _ in range(steps):
        evaluate(x, J, F)
        ws, st = mg.newton_step(J, F, x, 0.0, state, workspace=ws, status=st)
        got.append(x.cpu().numpy())
    tol = {1: 1e-10, 2: 1e-26, 4: 1e-56}[L]
    for k, (g, w) in enumerate(zip(got, want)):
        assert rel(orc, g, w) <= tol, k
    s = state.read()
    assert s["done"] == 0 and s["iterations"] == steps
    assert s["dx_norm"][0] > 1e-5 and s["dx_norm"][-1] < 1e3 * tol
    assert rel(orc, got[-1], xs) <= 1e3 * tol


def test_gate_stops_after_convergence(orc):
    """With tol > 0 the run stops itself; further steps leave x bit for bit unchanged."""
    import torch

    import paper_1210_0800_gb300 as mg

    m, n, L = 30, 24, 2
    A, c, b, xs = npb.problem(orc, m, n, L, 7400)
    dev = torch.device("cuda:0")
    x = torch.from_numpy(_start(xs, 7401)).to(dev)

    def evaluate(xd, J, F):
        Jh, Fh = npb.evaluate(orc, A, c, b, xd.cpu().numpy())
        J.copy_(torch.from_numpy(Jh))
        F.copy_(torch.from_numpy(Fh))

    s = mg.newton_corrector(evaluate, x, m, tol=1e-20, max_iter=12)
    assert s["done"] == 1
    assert 3 <= s["iterations"] < 12
    assert s["dx_norm"][-1] <= 1e-20 * s["x_norm"][-1]
    assert rel(orc, x.cpu().numpy(), xs) <= 1e-24
    # the state is the gate: a further step on a converged run changes nothing
    state = mg.NewtonState(dev)
    raw = np.zeros(mg.newton.STATE_BYTES, dtype=np.uint8)
    raw[:16] = np.array([1, 5, 0, 0], dtype=np.int32).view(np.uint8)
    state.buf.copy_(torch.from_numpy(raw))
    before = x.clone()
    J = torch.empty(A.shape, dtype=torch.float64, device=dev)
    F = torch.empty(b.shape, dtype=torch.float64, device=dev)
    evaluate(x, J, F)
    mg.newton_step(J, F, x, 0.0, state)
    assert torch.equal(x, before)
    assert state.read()["iterations"] == 5


def test_rank_deficient_jacobian_stops_the_run(orc):
    import torch

    import paper_1210_0800_gb300 as mg

    m, n, L = 20, 10, 2
    A, c, b, xs = npb.problem(orc, m, n, L, 7500)
    dev = torch.device("cuda:0")
    x = torch.from_numpy(_start(xs, 7501)).to(dev)
    before = x.clone()

    def evaluate(xd, J, F):
        Jh, Fh = npb.evaluate(orc, A, c, b, xd.cpu().numpy())
        Jh[3] = 0.0  # a zero column: r_33 = 0
        J.copy_(torch.from_numpy(Jh))
        F.copy_(torch.from_numpy(Fh))

    s = mg.newton_corrector(evaluate, x, m, tol=0.0, max_iter=3)
    assert s["done"] == 2 and s["status"] == 2 and s["iterations"] == 0
    assert torch.equal(x, before)


def test_graph_captured_run_matches_eager(orc):
    """A run whose evaluations are device copies (as in path tracking with the Jacobians
    evaluated on the GPU) captured in one CUDA graph: no host synchronisation inside, and
    the same iterates as the eager run."""
    import torch

    import paper_1210_0800_gb300 as mg

    m, n, L = 36, 28, 2
    A, c, b, xs = npb.problem(orc, m, n, L, 7600)
    x0 = _start(xs, 7601)
    steps = 5
    # the caller's evaluations along the oracle's iterates, resident on the device
    dev = torch.device("cuda:0")
    evals, x = [], x0.copy()
    for _ in range(steps):
        J, F = npb.evaluate(orc, A, c, b, x)
        evals.append((torch.from_numpy(J).to(dev), torch.from_numpy(F).to(dev)))
        x, _, _, _ = orc.newton_step(J, F, x)
    Jd = torch.empty(A.shape, dtype=torch.float64, device=dev)
    Fd = torch.empty(b.shape, dtype=torch.float64, device=dev)

    def run(xd, state, ws, st, stream):
        for i in range(steps):
            Jd.copy_(evals[i][0], non_blocking=True)
            Fd.copy_(evals[i][1], non_blocking=True)
            mg.newton_step(Jd, Fd, xd, 0.0, state, workspace=ws, status=st, stream=stream)

    ws = torch.empty(mg.newton.workspace_bytes(L, m, n), dtype=torch.uint8, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    xe = torch.from_numpy(x0.copy()).to(dev)
    se = mg.NewtonState(dev)
    run(xe, se, ws, st, torch.cuda.current_stream())  # also the first-call set-up, outside the capture
    torch.cuda.synchronize()

    xg = torch.from_numpy(x0.copy()).to(dev)
    sg = mg.NewtonState(dev)
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        run(xg, sg, ws, st, side)
    xg.copy_(torch.from_numpy(x0.copy()))
    sg.reset()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(xg, xe)
    a, e = sg.read(), se.read()
    assert a["iterations"] == e["iterations"] == steps
    assert np.array_equal(a["dx_norm"], e["dx_norm"])
