"""The benchmark's host logic for N > 1 ranks, run as two gloo processes on the CPU: the
slowest rank's time is the job's, replicas solve distinct systems, and only rank 0 of
the reference arm does any work."""

import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    mine = [10.0 + rank, 5.0 - rank, 7.0 * (rank + 1)]
    got = bench.max_over_ranks(mine, torch.device("cpu"), world)
    seeds = [bench.replica_seed("c1_qd_320x256", rank, i) for i in range(4)]
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    # the reference arm: ranks other than 0 return at once, without work or output
    cfg, unit = bench.workload_config("c1_qd_320x256", world)
    rc = bench.run_reference(type("A", (), {"steps": 1, "warmup": 0, "gpus": world,
                                            "workload": "c1_qd_320x256"})(), cfg, unit, rank, world) \
        if rank != 0 else 0
    dist.destroy_process_group()
    out[rank] = (got, gathered, rc)


@pytest.mark.timeout(120)
def test_two_rank_reduction_and_seeds():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(100)
            assert p.exitcode == 0
        res = dict(out)
    want = [11.0, 5.0, 14.0]
    for r in range(world):
        got, gathered, rc = res[r]
        assert got == want
        assert rc == 0
        a, b = gathered
        assert not set(a) & set(b)  # replicas solve distinct systems
