"""Phase timeline of one single-system solve (a diagnostic).

The kernels compiled with -DMGS_TRACE=1 record, per CTA, a global-timer stamp at each
phase boundary of every elimination step, the SM they ran on, and stamps of the
normalisation and back-substitution phases.  This module builds that variant of the
library (lib/trace/), runs a few solves of one size and prints where the time goes.

    python -m paper_1210_0800_gb300.trace LIMBS M N      (MGS_KERNEL, MGS_ROWS apply)

Phases of the grid-barrier kernel, per step k: reduction of the Br partial Gram rows,
coefficient division, look-ahead update of column k+1, update of the other columns,
wait for and copy of pivot k+1, partials of step k+1, grid barrier.  Of the cluster
schedule: the critical phases (a pivot applied to the next column a cluster publishes:
on the owner of column k+1, and ahead of it on the owner of column k+2), then per bulk
phase its Gram partials, cluster barrier and reduction, coefficient division, R/y stores
and updates, and the wait for and copy of the next pivot.  Each phase is the per-step mean
over the CTAs that ran it, summed over the steps.
"""

from __future__ import annotations

import ctypes
import sys

import numpy as np

from . import _binding, build, inputs

GRID_PHASES = ["reduce", "coef", "lookahead", "update", "wait+copy", "partials", "barrier"]
CLUSTER_PHASES = ["critical phases", "bulk partials", "barrier+reduce", "coef", "store+update", "pivot wait+copy"]


def _load_trace_library():
    lib = _binding.load(build.build(trace=True))
    lib.mgs_trace_layout.restype = ctypes.c_int
    lib.mgs_trace_layout.argtypes = [ctypes.c_int] * 4 + [ctypes.POINTER(ctypes.c_size_t),
                                                          ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    _binding._lib = lib  # the binding's calls below go to the trace variant
    return lib


def record(L: int, m: int, n: int, reps: int = 3, seed: int = 555):
    """Run `reps` solves of one size with the trace variant; returns (plan, stamps) with
    stamps[step, cta, slot] in nanoseconds (step n + 1 holds the epilogue stamps)."""
    import torch

    import paper_1210_0800_gb300 as mg

    lib = _load_trace_library()
    off, steps, ctas = ctypes.c_size_t(), ctypes.c_int(), ctypes.c_int()
    if lib.mgs_trace_layout(L, m, n, 1, ctypes.byref(off), ctypes.byref(steps), ctypes.byref(ctas)) != 0:
        raise RuntimeError("no layout for limbs=%d m=%d n=%d" % (L, m, n))
    plan = mg.mgs_plan_query(L, m, n, True)
    dev = torch.device("cuda:0")
    fn = {1: mg.ls_solve_d, 2: mg.ls_solve_dd, 4: mg.ls_solve_qd}[L]
    ws = torch.zeros(mg.mgs_workspace_bytes(L, m, n, True), dtype=torch.uint8, device=dev)
    nbytes = 8 * 8 * steps.value * ctas.value
    for rep in range(reps):
        A, _, b = inputs.system(m, n, L, seed + rep)
        ws[off.value: off.value + nbytes].zero_()
        fn(torch.from_numpy(A).to(dev), torch.from_numpy(b).to(dev), workspace=ws)
        torch.cuda.synchronize()
    raw = ws[off.value: off.value + nbytes].cpu().numpy().view(np.uint64)
    return plan, raw.reshape(steps.value, ctas.value, 8).astype(np.int64)


def summarize(plan, tr) -> str:
    """Per-phase sums of the per-step means over the CTAs active in the step."""
    nc = tr.shape[0] - 1
    sid = tr[0, :, 7]
    lines = ["plan %s" % plan,
             "CTAs %d on %d distinct SMs" % (len(sid), len(np.unique(sid)))]
    grid = plan["kernel"] == "grid"
    names = GRID_PHASES if grid else CLUSTER_PHASES
    tot = np.zeros(len(names))
    for k in range(nc - 1 if grid else nc):
        row = tr[k]
        act = row[:, 0] > 0
        if grid:
            if not act.any():
                continue
            for i in range(len(names)):
                end = tr[k + 1, act, 0] if i == len(names) - 1 else row[act, i + 1]
                tot[i] += np.mean(end - row[act, i])
        else:
            # stamps of step k: 1/5 start/end of a critical phase with pivot k; 0 bulk start,
            # 6 after its partials (0 where it had none), 2 after the cluster reduction,
            # 3 after the coefficients, 4 bulk end; 7 (k >= 1) pivot k received
            cr = (row[:, 1] > 0) & (row[:, 5] > 0)
            if cr.any():
                tot[0] += np.mean(row[cr, 5] - row[cr, 1])
            bk = (row[:, 0] > 0) & (row[:, 4] > 0)
            if bk.any():
                r = row[bk]
                mid = np.where(r[:, 6] > 0, r[:, 6], r[:, 0])
                tot[1] += np.mean(mid - r[:, 0])
                tot[2] += np.mean(r[:, 2] - mid)
                tot[3] += np.mean(r[:, 3] - r[:, 2])
                tot[4] += np.mean(r[:, 4] - r[:, 3])
            if k >= 1:
                prev = tr[k - 1]
                waits = []
                for c in np.nonzero(row[:, 7] > 0)[0]:
                    before = [v for v in (prev[c, 4], prev[c, 5]) if 0 < v < row[c, 7]]
                    if before:
                        waits.append(row[c, 7] - max(before))
                if waits:
                    tot[5] += float(np.mean(waits))
    first = tr[0, :, :7]
    t0 = first[first > 0].min()
    ep = tr[nc]
    lines.append("sweep %.1f us, solve %.1f us" % ((ep[:, 0].max() - t0) / 1e3, (ep[:, 3].max() - t0) / 1e3))
    for nm, v in zip(names, tot):
        lines.append("  %-16s %9.1f us" % (nm, v / 1e3))
    lines.append("  square roots %.1f us, Q and R scaling %.1f us, back substitution %.1f us" % (
        np.mean(ep[:, 1] - ep[:, 0]) / 1e3, np.mean(ep[:, 2] - ep[:, 1]) / 1e3, np.mean(ep[:, 3] - ep[:, 2]) / 1e3))
    return "\n".join(lines)


def main(argv=None) -> int:
    argv = sys.argv[1:] if argv is None else argv
    L, m, n = (int(a) for a in argv[:3])
    print(summarize(*record(L, m, n)))
    return 0


if __name__ == "__main__":
    sys.exit(main())
