"""The single-system kernels against the oracle on the same inputs: the cluster schedule
(no grid barrier per step) on hardware thread-block clusters and on software groups, and
the grid-barrier kernel; across the layouts that select them: one to eight row blocks per
cluster, more row blocks than a cluster holds, one and several columns per CTA, ragged
last row block."""

import os

import numpy as np
import pytest

from helpers import TOL, compare_ls, gpu_ls_solve, gpu_qr, planted_system, rel, upper
from paper_1210_0800_gb300 import inputs, mgs_plan_query

pytestmark = pytest.mark.gpu


@pytest.fixture(params=["default", "cluster", "group", "grid"])
def kernel(request, monkeypatch):
    if request.param == "default":
        monkeypatch.delenv("MGS_KERNEL", raising=False)
    else:
        monkeypatch.setenv("MGS_KERNEL", request.param)
    return request.param


# (m, n, L): Br = ceil(m / h) spans 1..8 and beyond (h = 64 unless shared memory forces
# a smaller block)
SHAPES = [(64, 64, 2), (65, 64, 2), (200, 150, 2), (320, 128, 2), (511, 60, 2), (600, 40, 2), (96, 96, 4),
          (150, 100, 4), (300, 31, 1)]


@pytest.mark.parametrize("m,n,L", SHAPES)
def test_kernel_vs_oracle(orc, kernel, m, n, L):
    plan = mgs_plan_query(L, m, n, True)
    if kernel == "default":
        assert plan["kernel"] in (("cluster", "grid") if L <= 2 and plan["Br"] <= 8 else ("grid",))
    elif kernel == "cluster" and plan["Br"] > 8:
        assert plan["kernel"] == "grid"
    else:
        assert plan["kernel"] == kernel
    A, _, b = planted_system(m, n, L, 4400 + 7 * m + n + L, orc=orc)
    compare_ls(orc, A, b)


@pytest.mark.parametrize("m,n,L", [(130, 100, 2), (70, 70, 4)])
def test_kernel_qr_vs_oracle(orc, kernel, m, n, L):
    A = inputs.matrix_uniform(m, n, L, 5300 + m + L)
    Qg, Rg, st = gpu_qr(A.copy())
    Qo, Ro, sto = orc.qr(A.copy())
    assert st == 0 and sto == 0
    assert rel(orc, Qg, Qo) <= TOL[L]
    assert rel(orc, upper(Rg), upper(Ro)) <= TOL[L]


def test_kernel_qr_last_column_zero(kernel):
    """A zero last column makes R singular: the plain QR reports MGS_ERANK."""
    A = inputs.matrix_uniform(100, 40, 2, 5401)
    A[39] = 0.0
    _, _, st = gpu_qr(A)
    assert st == 2


def test_kernel_rank_deficient_middle(kernel):
    A, _, b = inputs.system(150, 60, 2, 5402)
    A[30] = 0.0
    assert gpu_ls_solve(A, b)["status"] == 2


def test_kernels_agree(orc, monkeypatch):
    """All kernels reach the oracle's tolerance on one system, so they agree with each
    other to twice that; each is bitwise repeatable."""
    A, _, b = planted_system(256, 200, 2, 5500, orc=orc)
    res = {}
    for k in ("cluster", "group", "grid"):
        monkeypatch.setenv("MGS_KERNEL", k)
        res[k] = gpu_ls_solve(A.copy(), b.copy())
        again = gpu_ls_solve(A.copy(), b.copy())
        assert res[k]["status"] == 0
        assert np.array_equal(res[k]["x"], again["x"]) and np.array_equal(res[k]["R"], again["R"]), k
    for k in ("group", "grid"):
        assert rel(orc, res["cluster"]["x"], res[k]["x"]) <= 2 * TOL[2]
        assert rel(orc, upper(res["cluster"]["R"]), upper(res[k]["R"])) <= 2 * TOL[2]


@pytest.mark.parametrize("kk", ["grid", "cluster", "group"])
@pytest.mark.parametrize("m,n,L", [(65, 64, 2), (200, 150, 2), (96, 96, 4), (300, 31, 1)])
def test_256_threads_vs_oracle(orc, monkeypatch, kk, m, n, L):
    """Each kernel with 256 threads per CTA (two warps per SM sub-partition), the layout
    the plan picks when a CTA owns many columns."""
    monkeypatch.setenv("MGS_KERNEL", kk)
    monkeypatch.setenv("MGS_CTA_THREADS", "256")
    assert mgs_plan_query(L, m, n, True)["threads"] == 256
    A, _, b = planted_system(m, n, L, 4500 + 7 * m + n + L, orc=orc)
    compare_ls(orc, A, b)


def test_default_threads_follow_columns_per_cta(monkeypatch):
    monkeypatch.delenv("MGS_CTA_THREADS", raising=False)
    monkeypatch.delenv("MGS_KERNEL", raising=False)
    for (m, n, L) in [(320, 256, 4), (512, 512, 2), (32, 32, 2)]:
        p = mgs_plan_query(L, m, n, True)
        w = -(-(n + 1) // p["Bc"])
        assert p["threads"] == (256 if w >= 16 else 128), (m, n, p)
