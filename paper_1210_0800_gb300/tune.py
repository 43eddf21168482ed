"""Autotuner of the batched solve's launch shape (threads per CTA, CTAs per SM).

For a batch it times every candidate shape with CUDA events on the caller's stream
(each candidate on fresh copies of the inputs, since a solve overwrites them) and keeps
the fastest.  Results are cached in a JSON file keyed by device, precision and a bucket of
the batch's shape, so later batches of the same kind skip the search.
"""

from __future__ import annotations

import json
import os

CANDIDATES = [(128, 1), (128, 2), (128, 3), (256, 1), (256, 2)]
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "tune_cache.json")


def _bucket(v: int) -> int:
    b = 1
    while b < v:
        b *= 2
    return b


def cache_key(device_name: str, limbs: int, batch: int, max_n: int) -> str:
    return "%s|L%d|batch%d|n%d" % (device_name, limbs, _bucket(batch), _bucket(max_n))


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _clone(bt):
    from ._binding import Batch

    return Batch(bt.A_pool.clone(), bt.b_pool.clone(), bt.x_pool.clone(), bt.a_off, bt.b_off, bt.x_off, bt.m, bt.n,
                 bt.max_m, bt.max_n, bt.order)


def tune_batched(bt, reps: int = 2, cache_path: str | None = DEFAULT_CACHE, force: bool = False):
    """Return the fastest (threads, ctas_per_sm) for batch `bt` (and the timings)."""
    import torch

    from ._binding import ls_solve_batched

    name = torch.cuda.get_device_name(bt.A_pool.device)
    key = cache_key(name, bt.limbs, bt.batch, bt.max_n)
    cache = _load(cache_path) if cache_path else {}
    if not force and key in cache:
        return tuple(cache[key]["best"]), cache[key].get("ms", {})
    stream = torch.cuda.current_stream(bt.A_pool.device)
    times = {}
    for cand in CANDIDATES:
        best = None
        for _ in range(reps + 1):
            work = _clone(bt)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ls_solve_batched(work, tune=cand)
            e1.record(stream)
            e1.synchronize()
            t = e0.elapsed_time(e1)
            best = t if best is None else min(best, t)
        times["%d,%d" % cand] = best
    best = min(CANDIDATES, key=lambda c: times["%d,%d" % c])
    if cache_path:
        cache[key] = {"best": list(best), "ms": times}
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return best, times
