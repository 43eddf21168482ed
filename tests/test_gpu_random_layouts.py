"""Random sizes and launch layouts against the oracle: each case draws the precision, m,
n, the kernel (default, grid, cluster, group), the threads per CTA and the rows per row
block, so that the combinations of Br, Bc, ragged row blocks and columns per CTA the plan
can produce are exercised beyond the fixed shapes of the other tests."""

import random

import pytest

from helpers import compare_ls, planted_system

pytestmark = pytest.mark.gpu

_rng = random.Random(20261203)
CASES = []
for _t in range(36):
    _L = _rng.choice([1, 2, 2, 4])
    _m = _rng.randint(1, {1: 300, 2: 160, 4: 96}[_L])
    CASES.append((_t, _L, _m, _rng.randint(1, _m), _rng.choice([None, "grid", "cluster", "group"]),
                  _rng.choice([None, None, "256"]), _rng.choice([None, None, "32", "128"])))


@pytest.mark.parametrize("t,L,m,n,kernel,threads,rows", CASES)
def test_random_layout_vs_oracle(orc, monkeypatch, t, L, m, n, kernel, threads, rows):
    import torch

    from paper_1210_0800_gb300 import mgs_plan_query

    for var, val in (("MGS_KERNEL", kernel), ("MGS_CTA_THREADS", threads), ("MGS_ROWS", rows)):
        if val is None:
            monkeypatch.delenv(var, raising=False)
        else:
            monkeypatch.setenv(var, val)
    plan = mgs_plan_query(L, m, n, True)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert plan["Br"] * plan["Bc"] <= sms and plan["threads"] in (128, 256)
    A, _, b = planted_system(m, n, L, 778000 + t, orc=orc)
    compare_ls(orc, A, b)
