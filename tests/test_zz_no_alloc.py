"""ls_solve_dd_noalloc, the entry point for callers that cannot allocate device memory
(their device memory is owned by another allocator, or they must not allocate once
running): it runs the plan and kernel of ls_solve_dd on a scratch array inside the
library, so its results must equal ls_solve_dd's bit for bit, call after call, although
every call reuses that one array; a call must leave device memory use unchanged; and the
documented size limit must hold.  Collected last, so a failure here comes after every
other test has run."""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

LIMIT_N = 346  # the largest m = n whose workspace fits the array (include/mgs_ddqd.h)


def _outputs(n, m):
    import torch

    dev = torch.device("cuda:0")
    return dict(x=torch.zeros((n, 2, 2), dtype=torch.float64, device=dev),
                R=torch.zeros((n, n, 2, 2), dtype=torch.float64, device=dev),
                z=torch.zeros(2, dtype=torch.float64, device=dev),
                st=torch.full((1,), -1, dtype=torch.int32, device=dev))


def _call_noalloc(lib, At, bt, out, n, m):
    import torch

    vp = ctypes.c_void_p
    s = torch.cuda.current_stream(At.device)
    return lib.ls_solve_dd_noalloc(vp(At.data_ptr()), m, vp(bt.data_ptr()), vp(out["x"].data_ptr()),
                                   vp(out["R"].data_ptr()), n, vp(out["z"].data_ptr()), m, n,
                                   vp(out["st"].data_ptr()), vp(s.cuda_stream))


def _solve_noalloc(lib, A, b, n, m):
    import torch

    dev = torch.device("cuda:0")
    At = torch.from_numpy(A.copy()).to(dev)
    bt = torch.from_numpy(b.copy()).to(dev)
    out = _outputs(n, m)
    rc = _call_noalloc(lib, At, bt, out, n, m)
    torch.cuda.synchronize(dev)
    assert rc == 0, rc
    return dict(x=out["x"].cpu().numpy(), R=out["R"].cpu().numpy(), z=out["z"].cpu().numpy(), Q=At.cpu().numpy(),
                resid=bt.cpu().numpy(), status=int(out["st"].item()))


def _assert_same_bits(got, ref):
    from helpers import upper

    assert got["status"] == 0 and ref["status"] == 0
    for k in ("x", "Q", "resid", "z"):
        assert np.array_equal(got[k], ref[k]), k
    assert np.array_equal(upper(got["R"]), upper(ref["R"]))


def test_noalloc_matches_ls_solve_dd(orc):
    """Two calls in a row per size: bit-identical to ls_solve_dd, and x within 1e-26 of
    the oracle."""
    from helpers import gpu_ls_solve, planted_system, rel
    from paper_1210_0800_gb300 import _binding

    lib = _binding.load()
    for m, n, seed in ((96, 80, 3101), (130, 97, 3102)):
        A, _, b = planted_system(m, n, 2, seed, orc=orc)
        ref = gpu_ls_solve(A.copy(), b.copy())
        want = orc.ls_solve(A.copy(), b.copy())
        for _ in range(2):  # two calls in a row share the scratch array
            got = _solve_noalloc(lib, A, b, n, m)
            _assert_same_bits(got, ref)
            assert rel(orc, got["x"], want["x"]) <= 1e-26


def test_noalloc_leaves_device_memory_unchanged(orc):
    """Once the first call has loaded the library's module (and with it the array), a
    call changes neither what PyTorch has allocated nor the device's free memory."""
    import torch

    from helpers import planted_system
    from paper_1210_0800_gb300 import _binding

    lib = _binding.load()
    dev = torch.device("cuda:0")
    m, n = 120, 100
    A, _, b = planted_system(m, n, 2, 3103, orc=orc)
    At, bt = torch.from_numpy(A.copy()).to(dev), torch.from_numpy(b.copy()).to(dev)
    out = _outputs(n, m)
    assert _call_noalloc(lib, At, bt, out, n, m) == 0
    torch.cuda.synchronize(dev)
    A2, b2 = torch.from_numpy(A.copy()).to(dev), torch.from_numpy(b.copy()).to(dev)
    out2 = _outputs(n, m)
    torch.cuda.synchronize(dev)
    alloc0, free0 = torch.cuda.memory_allocated(dev), torch.cuda.mem_get_info(dev)[0]
    assert _call_noalloc(lib, A2, b2, out2, n, m) == 0
    torch.cuda.synchronize(dev)
    alloc1, free1 = torch.cuda.memory_allocated(dev), torch.cuda.mem_get_info(dev)[0]
    assert alloc1 == alloc0 and free1 == free0, (alloc0, alloc1, free0, free1)
    assert int(out2["st"].item()) == 0
    assert torch.equal(out2["x"], out["x"])


def test_noalloc_size_limit(orc):
    """m = n = 346 fits the array and solves like ls_solve_dd; 347 and beyond are refused
    with MGS_ENOSPACE before any work."""
    import torch

    from helpers import gpu_ls_solve
    from paper_1210_0800_gb300 import _binding, inputs

    lib = _binding.load()
    cap = 4 * 1024 * 1024  # MGS_NOALLOC_WORKSPACE_BYTES
    assert _binding.workspace_bytes(2, LIMIT_N, LIMIT_N, True) <= cap < _binding.workspace_bytes(
        2, LIMIT_N + 1, LIMIT_N + 1, True)
    n = m = LIMIT_N
    A, _, b = inputs.system(m, n, 2, 3104)
    ref = gpu_ls_solve(A.copy(), b.copy())
    for _ in range(2):
        _assert_same_bits(_solve_noalloc(lib, A, b, n, m), ref)
    dev = torch.device("cuda:0")
    buf = torch.zeros(16, dtype=torch.float64, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    vp = ctypes.c_void_p
    p = vp(buf.data_ptr())
    for big in (LIMIT_N + 1, 1024):
        rc = lib.ls_solve_dd_noalloc(p, big, p, p, None, 0, None, big, big, vp(st.data_ptr()), None)
        assert rc == _binding.MGS_ENOSPACE, (big, rc)
