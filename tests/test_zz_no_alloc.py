"""ls_solve_dd_noalloc, the entry point for callers that cannot allocate device memory:
it must give what ls_solve_dd gives, call after call, although every call reuses the one
scratch array inside the library.  Collected last, so a failure here comes after every
other test has run."""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _solve_noalloc(lib, A, b, n, m):
    import torch

    dev = torch.device("cuda:0")
    At = torch.from_numpy(A.copy()).to(dev)
    bt = torch.from_numpy(b.copy()).to(dev)
    x = torch.zeros((n, 2, 2), dtype=torch.float64, device=dev)
    R = torch.zeros((n, n, 2, 2), dtype=torch.float64, device=dev)
    z = torch.zeros(2, dtype=torch.float64, device=dev)
    st = torch.full((1,), -1, dtype=torch.int32, device=dev)
    s = torch.cuda.current_stream(dev)
    vp = ctypes.c_void_p
    rc = lib.ls_solve_dd_noalloc(vp(At.data_ptr()), m, vp(bt.data_ptr()), vp(x.data_ptr()), vp(R.data_ptr()), n,
                                 vp(z.data_ptr()), m, n, vp(st.data_ptr()), vp(s.cuda_stream))
    torch.cuda.synchronize(dev)
    assert rc == 0, rc
    return dict(x=x.cpu().numpy(), R=R.cpu().numpy(), z=z.cpu().numpy(), Q=At.cpu().numpy(),
                resid=bt.cpu().numpy(), status=int(st.item()))


def test_noalloc_matches_ls_solve_dd(orc):
    from helpers import gpu_ls_solve, planted_system, rel, upper
    from paper_1210_0800_gb300 import _binding

    lib = _binding.load()
    tol = 1e-26
    for m, n, seed in ((96, 80, 3101), (130, 97, 3102)):
        A, _, b = planted_system(m, n, 2, seed, orc=orc)
        ref = gpu_ls_solve(A.copy(), b.copy())
        assert ref["status"] == 0
        for _ in range(2):  # two calls in a row share the scratch array
            got = _solve_noalloc(lib, A, b, n, m)
            assert got["status"] == 0
            assert rel(orc, got["x"], ref["x"]) <= tol
            assert rel(orc, upper(got["R"]), upper(ref["R"])) <= tol
            assert rel(orc, got["Q"], ref["Q"]) <= tol
            assert abs(float(np.sum(got["z"])) - float(np.sum(ref["z"]))) <= tol * max(1.0, float(np.sum(ref["z"])))


def test_noalloc_rejects_oversize():
    import torch

    from paper_1210_0800_gb300 import _binding

    lib = _binding.load()
    dev = torch.device("cuda:0")
    buf = torch.zeros(16, dtype=torch.float64, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    vp = ctypes.c_void_p
    p = vp(buf.data_ptr())
    # n = 1024 needs far more than the built-in array: rejected before any work
    rc = lib.ls_solve_dd_noalloc(p, 1024, p, p, None, 0, None, 1024, 1024, vp(st.data_ptr()), None)
    assert rc == _binding.MGS_ENOSPACE
