"""Host-side logic on the CPU: the batched solve's hand-out orders, the tuner's shape
buckets, and the benchmark's contract that both arms describe the same workload."""

import numpy as np

import bench
from paper_1210_0800_gb300 import batch_order, inputs, tune


def _work(ms, ns):
    return np.asarray(ms, dtype=np.float64) * np.asarray(ns, dtype=np.float64) ** 2


def test_batch_orders_are_permutations():
    ms, ns = inputs.ragged_shapes(97, 4242, 16, 192, 0, 16)
    for kind in ("largest", "interleave"):
        o = batch_order(ms, ns, kind)
        assert o.dtype == np.int32 and sorted(o.tolist()) == list(range(97)), kind
    assert batch_order(ms, ns, "natural") is None and batch_order(ms, ns, None) is None


def test_largest_first_is_non_increasing_work():
    ms, ns = inputs.ragged_shapes(64, 4243, 16, 192, 0, 16)
    w = _work(ms, ns)[batch_order(ms, ns, "largest")]
    assert (np.diff(w) <= 0).all()


def test_interleave_alternates_largest_and_smallest():
    ms, ns = inputs.ragged_shapes(65, 4244, 16, 192, 0, 16)
    desc = batch_order(ms, ns, "largest")
    o = batch_order(ms, ns, "interleave")
    assert o[0] == desc[0] and o[1] == desc[-1] and o[2] == desc[1] and o[3] == desc[-2]
    # the first wave of half the systems holds about half the work of the largest-first one
    w = _work(ms, ns)
    half = len(o) // 2
    assert w[o[:half]].sum() < 0.75 * w[desc[:half]].sum()


def test_tuner_bucket_follows_the_size_distribution():
    ns_a = np.full(512, 100)
    ns_b = np.concatenate([np.full(256, 20), np.full(256, 180)])
    k_a = tune.cache_key("GB300", 2, 512, ns_a, 116)
    k_b = tune.cache_key("GB300", 2, 512, ns_b, 196)
    assert k_a != k_b
    # same bucket for batches that differ only inside the rounding
    assert tune.cache_key("GB300", 2, 500, ns_a + 3, 120) == tune.cache_key("GB300", 2, 512, ns_a, 116)
    assert tune.cache_key("GB300", 4, 512, ns_a, 116) != k_a


def test_tuner_labels():
    assert tune._label((256, 1, 2, 8), "largest") == "256,1,2,8,largest"


def test_both_bench_arms_share_the_config():
    for wl in list(bench.WORKLOADS) + list(bench.BATCHED) + list(bench.DIFF) + list(bench.NEWTON):
        cfg, unit = bench.workload_config(wl, 1)
        assert cfg["workload"] == wl and "l2" in cfg and "parallelism" in cfg
        assert unit.startswith(("systems/s", "Newton steps/s"))
    single = bench.single_config("c1_qd_320x256", 1)
    assert single == bench.workload_config("c1_qd_320x256", 1)[0]
    assert {"limbs", "m", "n", "extreme", "systems_per_step"} <= set(single)
    assert bench.single_config("c1_qd_320x256", 2)["parallelism"] != single["parallelism"]


def test_complex_mac_count():
    # m n (n + 1): the projections and updates of MGS on [A b] (n + 1 columns)
    assert bench.cmacs(4, 320, 256) == 320 * 256 * 257


def test_reference_steps_solve_the_gpu_arms_systems():
    """The reference arm's step i solves the system the GPU arm times at step i (rank 0)."""
    kind, L, A, b = bench._ref_problem("c1_qd_320x256", 7)
    A2, _, b2 = inputs.system(320, 256, 4, bench.replica_seed("c1_qd_320x256", 0, 7))
    assert kind == "solve" and L == 4 and np.array_equal(A, A2) and np.array_equal(b, b2)
