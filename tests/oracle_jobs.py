"""Oracle solves of the full-size workloads, run in worker processes while the GPU tests
run (the largest, quad double at m = n = 512, takes minutes on one core).

The pool is started from the collection hook in ``conftest.py`` with the ``spawn`` start
method, before any test touches the GPU; each job regenerates its inputs from the seeded
generators and returns the oracle's outputs.  Nothing here runs on the GPU.
"""

from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

# name -> (limbs of the problem, m, n, seed recipe, extreme, limbs the oracle computes in)
#   seed recipe: ("workload", name, index) -> inputs.system_seed(workload_seed(name), index)
#                ("plain", seed)           -> seed
FULLSIZE = {
    "c1_qd_320x256": (4, 320, 256, ("workload", "c1", 0), False, 4),
    "dd_256": (2, 256, 256, ("plain", 7702256), False, 2),
    "dd_512": (2, 512, 512, ("plain", 7702512), False, 2),
    "qd_512": (4, 512, 512, ("plain", 7704512), False, 4),
    "d_256": (1, 256, 256, ("plain", 7701256), False, 1),
    # the extreme-value DD workload: the DD oracle, the truth (the same stored numbers
    # solved at twice the limbs) and the complex-double solve of the leading limbs
    "c2_dd": (2, 256, 256, ("workload", "c2", 0), True, 2),
    "c2_truth": (2, 256, 256, ("workload", "c2", 0), True, 4),
    "c2_d": (2, 256, 256, ("workload", "c2", 0), True, 1),
}
# the extreme scaling in quad double at moderate sizes: QD oracle, L = 8 truth, DD solve
for _m, _n in ((64, 64), (90, 65), (160, 130)):
    for _lo in (4, 8, 2):
        FULLSIZE["qdx_%dx%d_L%d" % (_m, _n, _lo)] = (4, _m, _n, ("plain", 8800 + _m + _n), True, _lo)


def inputs_of(name):
    """(A, b) of a job, in the problem's own limbs."""
    from paper_1210_0800_gb300 import inputs

    L, m, n, recipe, extreme, _ = FULLSIZE[name]
    if recipe[0] == "workload":
        seed = inputs.system_seed(inputs.workload_seed(recipe[1]), recipe[2])
    else:
        seed = recipe[1]
    A, _, b = inputs.system(m, n, L, seed, extreme=extreme)
    return A, b


def relimb(X: np.ndarray, Lo: int) -> np.ndarray:
    """The same numbers with Lo limbs: padded with zero limbs, or cut to the leading Lo
    limbs (a cut changes the numbers; it is used only for the lower-precision solve)."""
    L = X.shape[-1]
    if Lo == L:
        return X.copy()
    if Lo > L:
        out = np.zeros(X.shape[:-1] + (Lo,), dtype=np.float64)
        out[..., :L] = X
        return out
    return np.ascontiguousarray(X[..., :Lo])


def solve(name):
    """Run the oracle's ls_solve of job `name`; returns its result dict."""
    import oracle

    A, b = inputs_of(name)
    Lo = FULLSIZE[name][5]
    return oracle.get().ls_solve(relimb(A, Lo), relimb(b, Lo))


class Jobs:
    """Handles of the submitted jobs: get(name) waits for one result."""

    def __init__(self, names):
        import oracle

        oracle.get()  # build the oracle here if it is missing or stale, not in every worker
        ctx = mp.get_context("spawn")
        procs = max(1, min(len(names), (os.cpu_count() or 2) - 2))
        self.pool = ctx.Pool(procs)
        # longest first, so the largest solve starts at once
        order = sorted(names, key=lambda k: -(FULLSIZE[k][1] * FULLSIZE[k][2] ** 2 * FULLSIZE[k][5] ** 2))
        self.res = {k: self.pool.apply_async(solve, (k,)) for k in order}

    def get(self, name, timeout=3000):
        return self.res[name].get(timeout)

    def close(self):
        self.pool.terminate()
        self.pool.join()
