"""Failure detection without a GPU fault: the solver kernels' bounded waits (the pivot-flag
wait and the grid barrier) are made to run out on a condition that never comes true.  The
wait records MGS_ETIMEOUT, raises the abort flag and returns; a wait that finds the abort
flag already raised falls through; the context stays usable for the next solve."""

import pytest

from helpers import compare_ls, planted_system
from paper_1210_0800_gb300 import mgs_wait_probe
from paper_1210_0800_gb300._binding import MGS_ETIMEOUT, MGS_OK

pytestmark = pytest.mark.gpu


def _words():
    import torch

    return torch.zeros(4, dtype=torch.int32, device="cuda")


@pytest.mark.parametrize("kind", [0, 1], ids=["flag_wait", "grid_barrier"])
def test_wait_runs_out(kind):
    words = _words()
    limit = 0.02
    secs = mgs_wait_probe(words, kind, limit)
    w = words.cpu().numpy()
    assert w[2] == MGS_ETIMEOUT and w[1] == 1
    assert limit <= secs < limit + 1.0, secs


@pytest.mark.parametrize("kind", [0, 1], ids=["flag_wait", "grid_barrier"])
def test_raised_abort_makes_waits_fall_through(kind):
    words = _words()
    words[1] = 1
    secs = mgs_wait_probe(words, kind, 2.0)
    w = words.cpu().numpy()
    assert w[2] == MGS_OK and w[1] == 1
    assert secs < 0.5, secs


def test_context_usable_after_a_timeout(orc):
    words = _words()
    mgs_wait_probe(words, 1, 0.01)
    assert int(words[2]) == MGS_ETIMEOUT
    A, _, b = planted_system(48, 40, 2, 9901, orc=orc)
    compare_ls(orc, A, b)
