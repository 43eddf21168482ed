"""Autotuner of the batched solve (one persistent launch over a ragged batch).

The tuned dimensions, per shape bucket of the batch:
  * threads per CTA and resident CTAs per SM;
  * the split: CTAs per system (a thread-block cluster sharing the rows of one system;
    rows per slice = m / split), or automatic;
  * chunks: the most lanes that share one (column, part) of a Gram row and update pass,
    i.e. the rows per lane (ceil(slice rows / chunks)) against the depth of the reduction
    trees;
  * the hand-out order of the work queue: largest systems first, or largest and smallest
    alternating (a first wave with about half the bytes in flight, which L2 can hold).
Every candidate is timed with CUDA events on the caller's stream, on fresh copies of the
inputs (a solve overwrites them); the search goes one dimension at a time from the
default, keeping the best of each stage.  Results are cached in a JSON file keyed by the
device, the precision, the batch size and the distribution of the system sizes (quartiles
of n, the largest m), so later batches of the same kind skip the search.
"""

from __future__ import annotations

import json
import os

SHAPES = [(128, 1), (128, 2), (128, 3), (256, 1), (256, 2)]  # (threads, CTAs per SM)
SPLITS = [1, 2, 4]
CHUNKS = [4, 8, 16]
ORDERS = ["largest", "interleave"]
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "tune_cache.json")


def _bucket(v: int) -> int:
    b = 1
    while b < v:
        b *= 2
    return b


def cache_key(device_name: str, limbs: int, batch: int, ns, max_m: int) -> str:
    """The shape bucket: batch rounded up to a power of two, the quartiles of n rounded up
    to multiples of 16, the largest m rounded up to a power of two."""
    import numpy as np

    q = [int(-(-int(v) // 16) * 16) for v in np.percentile(np.asarray(ns), [25, 50, 75, 100])]
    return "%s|L%d|batch%d|n%s|m%d" % (device_name, limbs, _bucket(batch), "-".join(map(str, q)), _bucket(max_m))


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _label(cand, order) -> str:
    return "%d,%d,%d,%d,%s" % (cand + (order,))


def tune_batched(bt, reps: int = 1, cache_path: str | None = DEFAULT_CACHE, force: bool = False):
    """Return (tune, order, times) for batch `bt`: tune = (threads, ctas_per_sm, split,
    chunks) for ls_solve_batched, order = the hand-out order ("largest" or "interleave",
    see Batch.set_order), times = {candidate label: ms}.  Leaves bt's order set to the
    winner."""
    import torch

    from ._binding import Batch, ls_solve_batched

    name = torch.cuda.get_device_name(bt.A_pool.device)
    ns = bt.n.cpu().numpy()
    key = cache_key(name, bt.limbs, bt.batch, ns, bt.max_m)
    cache = _load(cache_path) if cache_path else {}
    if not force and key in cache:
        best = tuple(cache[key]["best"])
        order = cache[key]["order"]
        bt.set_order(order)
        return best, order, cache[key].get("ms", {})
    stream = torch.cuda.current_stream(bt.A_pool.device)
    times = {}

    def run(cand, order):
        label = _label(cand, order)
        if label in times:
            return times[label]
        bt.set_order(order)
        best = None
        for _ in range(reps + 1):
            work = Batch(bt.A_pool.clone(), bt.b_pool.clone(), bt.x_pool.clone(), bt.a_off, bt.b_off, bt.x_off,
                         bt.m, bt.n, bt.max_m, bt.max_n, bt.order)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ls_solve_batched(work, tune=cand)
            e1.record(stream)
            e1.synchronize()
            t = e0.elapsed_time(e1)
            best = t if best is None else min(best, t)
        times[label] = best
        return best

    # stage by stage, each from the best so far
    cur, order = (256, 1, 0, 0), "largest"
    cands = [(t, c, 0, 0) for t, c in SHAPES]
    cur = min(cands, key=lambda cd: run(cd, order))
    cands = [cur] + [(cur[0], cur[1], s, 0) for s in SPLITS]
    cur = min(cands, key=lambda cd: run(cd, order))
    cands = [cur] + [(cur[0], cur[1], cur[2], ch) for ch in CHUNKS if ch <= cur[0]]
    cur = min(cands, key=lambda cd: run(cd, order))
    order = min(ORDERS, key=lambda o: run(cur, o))
    bt.set_order(order)
    if cache_path:
        cache[key] = {"best": list(cur), "order": order, "ms": times}
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return cur, order, times
