"""The C ABI's leading dimensions: A with lda > m and R with ldr > n give the same results
bit for bit as the contiguous layout, and the padding is left untouched."""

import ctypes

import numpy as np
import pytest

from paper_1210_0800_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L,m,n,pad_a,pad_r", [(2, 70, 50, 3, 5), (4, 40, 33, 1, 2), (1, 90, 64, 7, 1)])
def test_padded_leading_dimensions(L, m, n, pad_a, pad_r):
    import torch

    import paper_1210_0800_gb300 as mg
    from paper_1210_0800_gb300 import _binding

    A, _, b = inputs.system(m, n, L, 9300 + m)
    dev = torch.device("cuda:0")
    # contiguous reference through the binding
    Ac = torch.from_numpy(A.copy()).to(dev)
    bc = torch.from_numpy(b.copy()).to(dev)
    Rc = torch.zeros((n, n, 2, L), dtype=torch.float64, device=dev)
    fn = {1: mg.ls_solve_d, 2: mg.ls_solve_dd, 4: mg.ls_solve_qd}[L]
    xc, stc = fn(Ac, bc, R=Rc)
    # padded layouts through the C ABI: column j of A at j * lda elements, of R at j * ldr
    lda, ldr = m + pad_a, n + pad_r
    sentinel = -12345.0
    Ap = torch.full((n, lda, 2, L), sentinel, dtype=torch.float64, device=dev)
    Ap[:, :m] = torch.from_numpy(A)
    Rp = torch.full((n, ldr, 2, L), sentinel, dtype=torch.float64, device=dev)
    bp = torch.from_numpy(b.copy()).to(dev)
    xp = torch.empty((n, 2, L), dtype=torch.float64, device=dev)
    zp = torch.zeros(L, dtype=torch.float64, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = torch.empty(mg.mgs_workspace_bytes(L, m, n, True), dtype=torch.uint8, device=dev)
    lib = _binding.load()
    cfn = {1: lib.ls_solve_d, 2: lib.ls_solve_dd, 4: lib.ls_solve_qd}[L]
    vp = ctypes.c_void_p
    rc = cfn(vp(Ap.data_ptr()), lda, vp(bp.data_ptr()), vp(xp.data_ptr()), vp(Rp.data_ptr()), ldr,
             vp(zp.data_ptr()), m, n, vp(ws.data_ptr()), ctypes.c_size_t(ws.numel()), vp(st.data_ptr()),
             vp(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    assert int(st.item()) == 0 and int(stc.item()) == 0
    assert torch.equal(xp, xc)
    assert torch.equal(Ap[:, :m], Ac)
    assert torch.equal(bp, bc)
    for j in range(n):
        assert torch.equal(Rp[j, :j + 1], Rc[j, :j + 1])
    assert bool((Ap[:, m:] == sentinel).all())  # padding rows of A untouched
    assert bool((Rp[:, n:] == sentinel).all())  # padding rows of R untouched
