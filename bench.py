"""Benchmark: complex quad-double MGS least squares, m=320, n=256, a sequence of solves.

One step = one least-squares solve (MGS on [A b] + back substitution) of one system, on
the GPU, through the C ABI; the systems are distinct, pre-generated and resident in HBM
(a path tracker solving its Newton systems one after another).  The K timed systems
(5.3 MB each) are all distinct, so every step reads data that is not in L2 from the step
before (total far above the 129 MB L2).

Prints ONE JSON line (rank 0).  --impl reference times the CPU oracle instead: every step
solves in full the system the GPU arm times at that step, one process per host core.  Multi-GPU: replicas only
(the solves of a path are sequential; independent systems shard with no collective).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1210_0800_gb300 import inputs  # noqa: E402

METRIC = "systems/s and FP64-pipe % of peak, complex DD/QD MGS least squares"

WORKLOADS = {
    # name: (limbs, m, n, extreme)
    "c1_qd_320x256": (4, 320, 256, False),
    "c0_dd_32x32": (2, 32, 32, False),
    "c2_dd_256x256_extreme": (2, 256, 256, True),
    "dd_64": (2, 64, 64, False),
    "dd_128": (2, 128, 128, False),
    "dd_256": (2, 256, 256, False),
    "dd_512": (2, 512, 512, False),
    "qd_64": (4, 64, 64, False),
    "qd_128": (4, 128, 128, False),
    "qd_256": (4, 256, 256, False),
    "qd_512": (4, 512, 512, False),
    "d_32": (1, 32, 32, False),
    "d_128": (1, 128, 128, False),
    "d_256": (1, 256, 256, False),
}
DEFAULT = "c1_qd_320x256"
SWEEP = ["dd_64", "dd_128", "dd_256", "dd_512", "qd_64", "qd_128", "qd_256", "qd_512"]


# The paper's wall-clock seconds for 10,000 runs of MGS + one back substitution on m = n
# systems (Tesla C2050 and one core of a Xeon X5690): Table 4 (complex double) and
# Table 5 (complex double double, complex quad double).  Quoted as context only.
PAPER_TABLES = {
    1: {16: (2.01, 4.11), 32: (14.61, 6.52), 48: (47.80, 11.11), 64: (112.60, 15.38), 80: (217.52, 22.89),
        96: (373.06, 30.43), 112: (589.35, 40.82), 128: (876.11, 49.10), 144: (1243.26, 67.41),
        160: (1701.57, 80.42), 176: (2260.07, 99.94), 192: (2932.15, 116.90), 208: (3722.77, 149.45),
        224: (4641.71, 172.30), 240: (5703.77, 211.30), 256: (6935.10, 234.29)},
    2: {16: (17.17, 11.85), 32: (125.06, 22.44), 48: (408.20, 35.88), 64: (952.35, 55.18), 80: (1841.07, 79.11)},
    4: {16: (113.51, 143.07), 32: (813.65, 155.32), 48: (2556.36, 266.55), 64: (6216.06, 409.57),
        80: (12000.15, 597.47)},
}


def run_tables(args):
    """The sizes of the paper's Tables 4 and 5: per (limbs, n) the time of 10,000 solves
    on this GPU (distinct systems, inputs cold), one JSON line each, beside the paper's
    CPU and C2050 seconds."""
    import torch

    import paper_1210_0800_gb300 as mg

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    K, W = args.steps, args.warmup
    for L in (1, 2, 4):
        fn = {1: mg.ls_solve_d, 2: mg.ls_solve_dd, 4: mg.ls_solve_qd}[L]
        for n, (cpu_s, gpu_s) in sorted(PAPER_TABLES[L].items()):
            host = [inputs.system(n, n, L, inputs.system_seed(inputs.BASE_SEED + 5, i)) for i in range(K + W)]
            As = [torch.from_numpy(h[0]).to(dev) for h in host]
            bs = [torch.from_numpy(h[2]).to(dev) for h in host]
            x = torch.empty((n, 2, L), dtype=torch.float64, device=dev)
            ws = torch.empty(mg.mgs_workspace_bytes(L, n, n, True), dtype=torch.uint8, device=dev)
            st = torch.zeros(K + W, dtype=torch.int32, device=dev)
            for i in range(W):
                fn(As[i], bs[i], x=x, workspace=ws, status=st[i:i + 1])
            torch.cuda.synchronize(dev)
            flush_l2(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for i in range(W, K + W):
                fn(As[i], bs[i], x=x, workspace=ws, status=st[i:i + 1])
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1) / K
            ours_s = 10000 * ms / 1000.0
            print(json.dumps({
                "table": "Table 4" if L == 1 else "Table 5", "limbs": L, "m": n, "n": n,
                "ms_per_solve": ms, "seconds_per_10000": ours_s, "paper_c2050_seconds": gpu_s,
                "paper_cpu_seconds": cpu_s, "vs_c2050": gpu_s / ours_s,
                "status_errors": int((st != 0).sum().item())}))
    return 0


def hbm_bytes(L: int, m: int, n: int) -> int:
    """Algorithmic HBM bytes of one solve: [A b] read, Q and the residual column written,
    x and the upper triangle of R written."""
    e = 16 * L
    return e * (2 * m * (n + 1) + n + n * (n + 1) // 2)
# batched workloads: name -> (limbs, batch, n range, extra rows range)
BATCHED = {
    "c3_dd_batched_512": (2, 512, (16, 192), (0, 16)),
    "qd_batched_512": (4, 512, (16, 192), (0, 16)),
}

# FP64 pipe instructions of the kernels' primitives (static counts of csrc/ddqd.cuh):
# complex conjugated multiply-accumulate, complex update y -= c x, |x|^2 accumulate,
# complex / real division.
COST = {
    1: dict(mac=4, upd=4, norm=2, div=3),
    2: dict(mac=36, upd=42, norm=18, div=23),
    4: dict(mac=280, upd=322, norm=140, div=409),
}
# FP64 peak: 152 SMs x 4 sub-partitions x 0.5 FP64 lanes/clk (one DFMA warp-instruction
# per 64 cycles per sub-partition, measured) at the 2070 MHz maximum SM clock.
SMS, FP64_LANES_PER_CLK_SM = 152, 2.0


L2_FLUSH_BYTES = 256 << 20  # twice the 129 MB L2
L2_NOTE = ("every step solves its own distinct system(s), with inputs no earlier step touched (GPU arm: a %d MB "
           "write flushed L2 after setup and warm-up; only the workspace is reused across steps)"
           % (L2_FLUSH_BYTES >> 20))


def flush_l2(dev):
    import torch

    buf = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    buf.fill_(1)
    torch.cuda.synchronize(dev)
    del buf


def fp64_ops(L: int, m: int, n: int) -> float:
    """Algorithmic FP64 instructions (lane operations) of one solve."""
    c = COST[L]
    nc = n + 1
    pairs = nc * (nc - 1) / 2  # (pivot k, column j > k) of the augmented matrix
    bulk = pairs * m * (c["mac"] + c["upd"])
    norms = nc * m * c["norm"]
    qdiv = n * m * c["div"]
    backsub = n * (n - 1) / 2 * c["upd"] + n * c["div"]
    return bulk + norms + qdiv + backsub


def peak_fp64_ops_per_s(sm_max_mhz: float) -> float:
    return SMS * FP64_LANES_PER_CLK_SM * sm_max_mhz * 1e6


def kernel_source_sha() -> str:
    """Hash of the sources of the single-system solver kernels (the ncu traffic figure is
    valid for this hash only)."""
    import hashlib

    names = ["ddqd.cuh", "mgs_kernel.cuh", "mgs_cluster.cuh", "launch.cuh", "mgs_d.cu", "mgs_dd.cu", "mgs_qd.cu",
             "api.cu"]
    h = hashlib.sha256()
    for name in names:
        h.update(name.encode())
        with open(os.path.join(ROOT, "paper_1210_0800_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload: str):
    """DRAM bytes per launch from the committed ncu capture, or None when the kernel
    sources changed since that capture (or the workload was not captured)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    if t.get("kernel_source_sha") != kernel_source_sha():
        return None
    return t.get("traffic_bytes_per_launch", {}).get(workload)


def max_over_ranks(values, device, world):
    """Element-wise maximum over the ranks of per-rank timings: the slowest replica sets
    the job's time (barrier-bracketed timed regions on every rank)."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def replica_seed(workload: str, rank: int, index: int) -> int:
    """Seed of system `index` on `rank`: replicas solve distinct systems."""
    return inputs.system_seed(inputs.workload_seed(workload), rank * 100000 + index)


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(gpu_index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle arm
def shared_config(workload: str, world: int, **extra) -> dict:
    """The workload's config, identical in both arms (the oracle arm solves the same
    systems as the GPU's timed steps)."""
    cfg = {"workload": workload}
    cfg.update(extra)
    cfg["l2"] = L2_NOTE
    cfg["parallelism"] = ("replicas: one independent system per step on every GPU" if world > 1
                          else "one independent system per step")
    return cfg


def single_config(workload: str, world: int) -> dict:
    L, m, n, extreme = WORKLOADS[workload]
    return shared_config(workload, world, limbs=L, m=m, n=n, extreme=extreme, systems_per_step=1)


def batched_config(workload: str, world: int) -> dict:
    L, batch, n_rng, e_rng = BATCHED[workload]
    return shared_config(workload, world, limbs=L, systems_per_step=batch, n_range=list(n_rng),
                         m_minus_n_range=list(e_rng))


def diff_config(workload: str, world: int) -> dict:
    L, m, n, B = DIFF[workload]
    return shared_config(workload, world, limbs=L, m=m, n=n, systems_per_step=B,
                         step="forward solve + adjoint (dL/dA, dL/db for L = sum |x|^2)")


def newton_config(workload: str, world: int) -> dict:
    L, m, n, S = NEWTON[workload]
    return shared_config(workload, world, limbs=L, m=m, n=n, newton_steps_per_run=S)


def workload_config(workload: str, world: int):
    """(config, unit) of a workload, shared by both arms."""
    if workload in WORKLOADS:
        return single_config(workload, world), "systems/s"
    if workload in BATCHED:
        return batched_config(workload, world), "systems/s"
    if workload in DIFF:
        return diff_config(workload, world), "systems/s"
    return newton_config(workload, world), "Newton steps/s (one solve each)"


def cmacs(L: int, m: int, n: int) -> float:
    """Complex multiply-accumulates of the projections and updates of one solve (the
    paper's operation count: m n (n + 1), half projections r_kj = q_k^H a_j, half updates
    a_j -= r_kj q_k over the augmented [A b]); independent of how a primitive is built."""
    return float(m) * n * (n + 1)


def _ref_problem(workload: str, index: int):
    """(kind, limbs, A, b) of the system the GPU arm times as step `index` (rank 0)."""
    if workload in WORKLOADS:
        L, m, n, extreme = WORKLOADS[workload]
        A, _, b = inputs.system(m, n, L, replica_seed(workload, 0, index), extreme=extreme)
        return "solve", L, A, b
    if workload in BATCHED:
        L, batch, n_rng, e_rng = BATCHED[workload]
        seed = inputs.system_seed(inputs.BASE_SEED + 3, 0)
        ms, ns = inputs.ragged_shapes(batch, seed, n_rng[0], n_rng[1], e_rng[0], e_rng[1])
        i = index % batch
        A, _, b = inputs.system(int(ms[i]), int(ns[i]), L, inputs.system_seed(seed, i))
        return "solve", L, A, b
    if workload in DIFF:
        L, m, n, B = DIFF[workload]
        A, _, b = inputs.system(m, n, L, replica_seed(workload, 0, index % B))
        return "adjoint", L, A, b
    L, m, n, S = NEWTON[workload]
    A, x0, b = inputs.system(m, n, L, replica_seed(workload, 0, index % S))
    return "newton", L, A, (b, x0)


def _ref_task(task):
    """One oracle step (a worker-process entry point): returns (seconds, status, what)."""
    workload, index = task
    import oracle

    o = oracle.get()
    kind, L, A, b = _ref_problem(workload, index)
    t0 = time.perf_counter()
    if kind == "solve":
        st = o.ls_solve(A, b)["status"]
    elif kind == "adjoint":
        r = o.ls_solve(A.copy(), b.copy())
        st = max(r["status"], o.ls_adjoint(A, b, 2.0 * r["x"])[3])
    else:
        st = o.newton_step(A, b[0], b[1])[3]
    dt = time.perf_counter() - t0
    return dt, st, "%s of a complex %s %dx%d system" % ({"solve": "ls_solve", "adjoint": "ls_solve + ls_adjoint",
                                                         "newton": "newton_step"}[kind],
                                                        {1: "D", 2: "DD", 4: "QD"}[L], A.shape[1], A.shape[0])


def _ref_warm(_):
    import oracle

    o = oracle.get()
    A, _, b = inputs.system(8, 8, 2, 1)
    o.ls_solve(A, b)
    return os.getpid()


def cpu_baseline(workload: str, count: int, first: int):
    """The oracle on this host, one core: `count` steps of the workload (the systems the
    GPU timed from index `first` on), each solved in full; returns the cpu_baseline entry
    (steps per second)."""
    total, what = 0.0, ""
    for i in range(count):
        dt, _, what = _ref_task((workload, first + i))
        total += dt
    return {"value": count / total, "unit": "systems/s" if workload not in NEWTON else "Newton steps/s",
            "cores": 1, "kind": "oracle",
            "sample": "%d full step%s on one core, each an oracle %s that the GPU arm also solves; %.1f s" % (
                count, "s" if count > 1 else "", what, total)}


def run_reference(args, config, unit, rank, world):
    """The oracle arm: every one of the K steps solves in full the system the GPU arm
    times at that step, one step per process, min(K, host cores) processes at a time;
    value = K / wall-clock seconds of the timed region."""
    if rank != 0:
        return 0
    import multiprocessing as mproc

    K, W = args.steps, args.warmup
    cores = os.cpu_count() or 1
    procs = max(1, min(K, cores))
    ctx = mproc.get_context("spawn")
    with ctx.Pool(procs) as pool:
        pool.map(_ref_warm, range(procs))  # workers up and the oracle loaded in each
        for i in range(W):  # warm-up steps: small systems, untimed
            pool.map(_ref_warm, range(procs))
        t0 = time.perf_counter()
        res = pool.map(_ref_task, [(args.workload, W + i) for i in range(K)], chunksize=1)
        wall = time.perf_counter() - t0
    secs = [r[0] for r in res]
    bad = sum(1 for r in res if r[1] != 0)
    value = K / wall
    desc = ("%d full steps, each the %s the GPU arm times at that step; %d processes on %d host cores; "
            "median %.3g s per step on one core" % (K, res[0][2], procs, cores, statistics.median(secs)))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": unit, "n_gpus": args.gpus,
        "steps": K, "warmup": W, "ms_per_step": 1000.0 * wall / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config,
        "cpu_baseline": {"value": value, "unit": unit, "cores": procs, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "reference_step": res[0][2] + (" (one system of each GPU step's batch)" if args.workload in BATCHED or
                                       args.workload in DIFF else
                                       " (one Newton step of a GPU run)" if args.workload in NEWTON else ""),
        "single_core_s_per_step": statistics.median(secs),
        "nproc": cores,
        "wall_s": wall,
        "status_errors": bad,
    }
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------- GPU arm
def run_gpu(args, L, m, n, extreme, rank, world):
    import torch

    import paper_1210_0800_gb300 as mg

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    fn = {1: mg.ls_solve_d, 2: mg.ls_solve_dd, 4: mg.ls_solve_qd}[L]
    K, W = args.steps, args.warmup
    total = K + W
    # distinct systems for every step (rank-dependent seeds: replicas solve different systems)
    seeds = [replica_seed(args.workload, rank, i) for i in range(total)]
    host = [inputs.system(m, n, L, s, extreme=extreme) for s in seeds]
    As = [torch.from_numpy(h[0]).to(dev) for h in host]
    bs = [torch.from_numpy(h[2]).to(dev) for h in host]
    xs = [torch.empty((n, 2, L), dtype=torch.float64, device=dev) for _ in range(total)]
    ws = torch.empty(mg.mgs_workspace_bytes(L, m, n, True), dtype=torch.uint8, device=dev)
    st = torch.zeros(total, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    for i in range(W):
        fn(As[i], bs[i], x=xs[i], workspace=ws, status=st[i:i + 1])
    torch.cuda.synchronize(dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush_l2(dev)
    clocks = ClockSampler(local)
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize(dev)
    t_start.record(stream)
    for i in range(K):
        j = W + i
        ev[i][0].record(stream)
        fn(As[j], bs[j], x=xs[j], workspace=ws, status=st[j:j + 1])
        ev[i][1].record(stream)
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clk = clocks.stop()
    ms_total = t_start.elapsed_time(t_end)
    per_solve_ms = [a.elapsed_time(b) for a, b in ev]
    statuses = st.cpu().numpy().tolist()
    bad = [s for s in statuses if s != 0]

    # end to end: pinned host buffers -> device, solve, x -> host, every step
    Ah = [torch.from_numpy(h[0]).pin_memory() for h in host[:min(total, 8)]]
    bh = [torch.from_numpy(h[2]).pin_memory() for h in host[:min(total, 8)]]
    xh = torch.empty((n, 2, L), dtype=torch.float64).pin_memory()
    Ad = torch.empty_like(As[0])
    bd = torch.empty_like(bs[0])
    xd = torch.empty_like(xs[0])
    Ke = max(3, min(K, 10))
    for i in range(2):
        Ad.copy_(Ah[i % len(Ah)], non_blocking=True)
        bd.copy_(bh[i % len(bh)], non_blocking=True)
        fn(Ad, bd, x=xd, workspace=ws, status=st[0:1])
        xh.copy_(xd, non_blocking=True)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(Ke):
        Ad.copy_(Ah[i % len(Ah)], non_blocking=True)
        bd.copy_(bh[i % len(bh)], non_blocking=True)
        fn(Ad, bd, x=xd, workspace=ws, status=st[0:1])
        xh.copy_(xd, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = e0.elapsed_time(e1) / Ke
    h2d = As[0].numel() * 8 + bs[0].numel() * 8
    d2h = xs[0].numel() * 8

    ms, e2e_ms = max_over_ranks([ms_total, e2e_ms], dev, world)
    if rank != 0:
        return 0

    value = world * K / (ms / 1000.0)
    kernel_ms = statistics.mean(per_solve_ms)
    ops = fp64_ops(L, m, n)
    peaks = read_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_ops = peak_fp64_ops_per_s(sm_max)
    achieved_ops = ops / (kernel_ms / 1000.0)
    line = {
        "metric": METRIC, "value": value, "unit": "systems/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": single_config(args.workload, world),
        "e2e": {"value": world / (e2e_ms / 1000.0), "unit": "systems/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": K,
        "roofline": {"bound": "alu", "achieved": 2 * achieved_ops / 1e12, "peak": 2 * peak_ops / 1e12,
                     "unit": "TFLOP/s", "frac": achieved_ops / peak_ops,
                     "traffic": measured_traffic(args.workload),
                     "note": "FP64 pipe: algorithmic FP64 instructions of the kernel's primitives per solve "
                             "(%.4g) / CUDA-event time per solve; each instruction counted as one FMA slot "
                             "(2 flops) like the peak (152 SMs x 2 DFMA/clk x %.0f MHz)" % (ops, sm_max)},
        "kernel_ms": kernel_ms,
        "cmac_rate": {"value": cmacs(L, m, n) / (kernel_ms / 1000.0) / 1e9, "unit": "G complex MAC/s",
                      "per_solve": cmacs(L, m, n),
                      "note": "m n (n + 1) complex multiply-accumulates of the projections and updates per "
                              "solve / CUDA-event time per solve; independent of the primitives' cost"},
        "hbm": {"bytes_per_solve": hbm_bytes(L, m, n), "achieved_gbs": hbm_bytes(L, m, n) / kernel_ms / 1e6,
                "note": "algorithmic bytes / kernel time; the solve is FP64-bound, not HBM-bound"},
        "status_errors": len(bad),
    }
    if clk:
        line["clocks"] = clk
    # the FP64 FMA rate measured on this GPU beside the derived peak the roofline uses
    probe = mg._binding.fp64_probe(blocks=4 * torch.cuda.get_device_properties(dev).multi_processor_count)
    line["roofline"]["measured_fp64_fma_per_s"] = probe
    line["roofline"]["measured_over_derived_peak"] = probe / peak_ops
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, 1, W)
    print(json.dumps(line))
    return 0


def run_gpu_batched(args, rank, world):
    """One step = one launch solving a ragged batch of independent systems (replayed from
    a CUDA graph); every step works on its own, distinct batch resident in HBM."""
    import torch

    import paper_1210_0800_gb300 as mg
    from paper_1210_0800_gb300 import tune as tuner

    L, batch, n_rng, e_rng = BATCHED[args.workload]
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    K, W = args.steps, args.warmup
    seed0 = inputs.BASE_SEED + 3
    host = inputs.ragged_batch(L, batch, n_rng, e_rng, inputs.system_seed(seed0, rank))
    ops = sum(fp64_ops(L, A.shape[1], A.shape[0]) for A, _ in host)
    # distinct device copies of the batch for warm-up + timed steps (pools are overwritten)
    base = mg.make_batch(host, dev)
    best, best_order, times = tuner.tune_batched(base, reps=1)
    batches = [mg.Batch(base.A_pool.clone(), base.b_pool.clone(), base.x_pool.clone(), base.a_off, base.b_off,
                        base.x_off, base.m, base.n, base.max_m, base.max_n, base.order) for _ in range(K + W)]
    need = mg._binding.batched_workspace_bytes(L, batch, base.max_m, base.max_n, best)
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    st = torch.zeros((K + W, batch), dtype=torch.int32, device=dev)
    # capture one graph per batch copy
    graphs = []
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        for i in range(K + W):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=side):
                mg.ls_solve_batched(batches[i], workspace=ws, status=st[i], tune=best)
            graphs.append(g)
    torch.cuda.current_stream(dev).wait_stream(side)
    torch.cuda.synchronize(dev)
    stream = torch.cuda.current_stream(dev)
    for i in range(W):
        graphs[i].replay()
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush_l2(dev)
    clocks = ClockSampler(local)
    time.sleep(0.3)
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
    torch.cuda.synchronize(dev)
    t0e.record(stream)
    for i in range(K):
        ev[i][0].record(stream)
        graphs[W + i].replay()
        ev[i][1].record(stream)
    t1e.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms_total = t0e.elapsed_time(t1e)
    kernel_ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    bad = int((st[W:] != 0).sum().item())
    # end to end: pinned host pools -> device, solve, x pool -> host
    Ah, bh = base.A_pool.cpu().pin_memory(), base.b_pool.cpu().pin_memory()
    xh = torch.empty_like(base.x_pool, device="cpu").pin_memory()
    work = batches[0]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    Ke = 3
    e0.record(stream)
    for _ in range(Ke):
        work.A_pool.copy_(Ah, non_blocking=True)
        work.b_pool.copy_(bh, non_blocking=True)
        mg.ls_solve_batched(work, workspace=ws, status=st[0], tune=best)
        xh.copy_(work.x_pool, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = e0.elapsed_time(e1) / Ke
    # the same systems solved one after another with the single-system solve
    fn = {1: mg.ls_solve_d, 2: mg.ls_solve_dd, 4: mg.ls_solve_qd}[L]
    nseq = min(batch, args.seq_sample)
    sel = list(range(0, batch, max(1, batch // nseq)))[:nseq]
    Ad = [torch.from_numpy(host[i][0]).to(dev) for i in sel]
    bd = [torch.from_numpy(host[i][1]).to(dev) for i in sel]
    torch.cuda.synchronize(dev)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for A_, b_ in zip(Ad, bd):
        fn(A_, b_)
    s1.record(stream)
    torch.cuda.synchronize(dev)
    seq_ms = s0.elapsed_time(s1)
    seq_ops = sum(fp64_ops(L, host[i][0].shape[1], host[i][0].shape[0]) for i in sel)
    ms_total, e2e_ms = max_over_ranks([ms_total, e2e_ms], dev, world)
    if rank != 0:
        return 0
    value = world * batch * K / (ms_total / 1000.0)
    peaks = read_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_ops = peak_fp64_ops_per_s(sm_max)
    achieved = ops / (kernel_ms / 1000.0)
    h2d = (base.A_pool.numel() + base.b_pool.numel()) * 8
    line = {
        "metric": METRIC, "value": value, "unit": "systems/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms_total / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": batched_config(args.workload, world),
        "launch": {"max_m": base.max_m, "max_n": base.max_n,
                   "how": "one persistent launch per step, replayed from a CUDA graph",
                   "tune": {"threads": best[0], "ctas_per_sm": best[1], "split": best[2], "chunks": best[3],
                            "order": best_order, "candidates_ms": times}},
        "e2e": {"value": world * batch / (e2e_ms / 1000.0), "unit": "systems/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": base.x_pool.numel() * 8},
        "gpu_launches": K,
        "roofline": {"bound": "alu", "achieved": 2 * achieved / 1e12, "peak": 2 * peak_ops / 1e12,
                     "unit": "TFLOP/s", "frac": achieved / peak_ops, "traffic": measured_traffic(args.workload),
                     "note": "FP64 pipe: algorithmic FP64 instructions of all systems (%.4g) per launch / "
                             "CUDA-event time per launch" % ops},
        "kernel_ms": kernel_ms,
        "cmac_rate": {"value": sum(cmacs(L, A.shape[1], A.shape[0]) for A, _ in host) / (kernel_ms / 1000.0) / 1e9,
                      "unit": "G complex MAC/s"},
        "sequential_plain": {"value": len(sel) / (seq_ms / 1000.0), "unit": "systems/s",
                             "systems": len(sel), "frac": (seq_ops / (seq_ms / 1000.0)) / peak_ops,
                             "note": "the same systems (every %d-th) solved one after another with the "
                                     "single-system solve on the same GPU" % max(1, batch // nseq)},
        "status_errors": bad,
    }
    if clk:
        line["clocks"] = clk
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, 8, 0)
    print(json.dumps(line))
    return 0


DIFF = {"c4_dd_diff_160x128x64": (2, 160, 128, 64)}
# Newton corrector runs: (limbs, m, n, steps per run)
NEWTON = {"newton_dd_256x256x8": (2, 256, 256, 8), "newton_qd_320x256x8": (4, 320, 256, 8)}


def run_gpu_newton(args, rank, world):
    """One step = one run of gated Newton corrector steps (newton_step_*) on device-resident
    Jacobians and residuals, as in path tracking with the evaluation on the GPU (the
    caller's: here copies of pre-generated J_i, F_i), the whole run replayed from one CUDA
    graph; beside it the same run launched eagerly and the plain solves it contains."""
    import torch

    import paper_1210_0800_gb300 as mg

    L, m, n, S = NEWTON[args.workload]
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    K, W = args.steps, args.warmup
    host = [inputs.system(m, n, L, replica_seed(args.workload, rank, i)) for i in range(S)]
    Js = [torch.from_numpy(h[0]).to(dev) for h in host]
    Fs = [torch.from_numpy(h[2]).to(dev) for h in host]
    x0 = torch.from_numpy(host[0][1]).to(dev)
    J = torch.empty_like(Js[0])
    F = torch.empty_like(Fs[0])
    x = x0.clone()
    ws = torch.empty(mg.newton.workspace_bytes(L, m, n), dtype=torch.uint8, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    state = mg.NewtonState(dev)

    def run(stream):
        for i in range(S):
            J.copy_(Js[i], non_blocking=True)
            F.copy_(Fs[i], non_blocking=True)
            mg.newton_step(J, F, x, 0.0, state, workspace=ws, status=st, stream=stream)

    cur = torch.cuda.current_stream(dev)
    run(cur)  # first-call set-up outside the capture
    torch.cuda.synchronize(dev)
    side = torch.cuda.Stream(dev)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        run(side)

    def replay():
        x.copy_(x0, non_blocking=True)
        state.buf.zero_()
        g.replay()

    for _ in range(W):
        replay()
    torch.cuda.synchronize(dev)
    flush_l2(dev)
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
    clocks = ClockSampler(local)
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(cur)
    for _ in range(K):
        replay()
    e1.record(cur)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / K
    done = state.read()
    # the same run launched eagerly, and the plain solves alone
    e0.record(cur)
    for _ in range(3):
        x.copy_(x0, non_blocking=True)
        state.buf.zero_()
        run(cur)
    e1.record(cur)
    torch.cuda.synchronize(dev)
    eager_ms = e0.elapsed_time(e1) / 3
    fn = {1: mg.ls_solve_d, 2: mg.ls_solve_dd, 4: mg.ls_solve_qd}[L]
    wss = torch.empty(mg.mgs_workspace_bytes(L, m, n, True), dtype=torch.uint8, device=dev)
    xs = torch.empty_like(x)
    e0.record(cur)
    for i in range(S):
        J.copy_(Js[i], non_blocking=True)
        F.copy_(Fs[i], non_blocking=True)
        fn(J, F, x=xs, workspace=wss, status=st)
    e1.record(cur)
    torch.cuda.synchronize(dev)
    solves_ms = e0.elapsed_time(e1)
    # end to end: x0 up, the run, the final x and the state down
    xh = torch.empty_like(x, device="cpu").pin_memory()
    x0h = x0.cpu().pin_memory()
    sh = torch.empty_like(state.buf, device="cpu").pin_memory()
    e0.record(cur)
    for _ in range(3):
        x.copy_(x0h, non_blocking=True)
        state.buf.zero_()
        g.replay()
        xh.copy_(x, non_blocking=True)
        sh.copy_(state.buf, non_blocking=True)
    e1.record(cur)
    torch.cuda.synchronize(dev)
    e2e_ms = e0.elapsed_time(e1) / 3
    ms, eager_ms, e2e_ms = max_over_ranks([ms, eager_ms, e2e_ms], dev, world)
    if rank != 0:
        return 0
    ops = S * fp64_ops(L, m, n)
    peaks = read_peaks()
    peak_ops = peak_fp64_ops_per_s(float(peaks.get("sm_max_mhz", 2070.0)))
    line = {
        "metric": METRIC, "value": world * S / (ms / 1000.0), "unit": "Newton steps/s (one solve each)",
        "n_gpus": world, "steps": K, "warmup": W, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": newton_config(args.workload, world),
        "step": "one CUDA-graph replay of %d gated newton_step calls, J and F copied in from device memory "
                "before each" % S,
        "e2e": {"value": world * S / (e2e_ms / 1000.0), "unit": "Newton steps/s",
                "h2d_bytes_per_step": x0h.numel() * 8, "d2h_bytes_per_step": xh.numel() * 8 + sh.numel()},
        "gpu_launches": 3 * S * K,
        "roofline": {"bound": "alu", "achieved": 2 * ops / (ms / 1000.0) / 1e12, "peak": 2 * peak_ops / 1e12,
                     "unit": "TFLOP/s", "frac": ops / (ms / 1000.0) / peak_ops, "traffic": None,
                     "note": "algorithmic FP64 instructions of the solves (%.4g) per run" % ops},
        "eager_run_ms": eager_ms,
        "plain_solves_ms": solves_ms,
        "corrector_overhead": (ms - solves_ms) / solves_ms,
        "state_after_run": {"done": done["done"], "iterations": done["iterations"]},
    }
    if clk:
        line["clocks"] = clk
    print(json.dumps(line))
    return 0


def run_gpu_diff(args, rank, world):
    """One step = forward solve of a batch of uniform systems plus the adjoint for
    L = sum |x|^2 (dL/dx = 2x), through the torch.autograd.Function."""
    import torch

    import paper_1210_0800_gb300 as mg

    L, m, n, B = DIFF[args.workload]
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    K, W = args.steps, args.warmup
    host = [inputs.system(m, n, L, replica_seed(args.workload, rank, i)) for i in range(B)]
    A0 = torch.from_numpy(np.stack([h[0] for h in host])).to(dev)
    b0 = torch.from_numpy(np.stack([h[2] for h in host])).to(dev)
    As = [A0.clone().requires_grad_(True) for _ in range(K + W)]
    bs = [b0.clone().requires_grad_(True) for _ in range(K + W)]
    stream = torch.cuda.current_stream(dev)

    def step(i):
        x = mg.lstsq(As[i], bs[i])
        x.backward(gradient=2.0 * x.detach())

    for i in range(W):
        step(i)
    torch.cuda.synchronize(dev)
    flush_l2(dev)
    clocks = ClockSampler(local)
    time.sleep(0.3)
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
    t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    t0e.record(stream)
    for i in range(K):
        step(W + i)
    t1e.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = t0e.elapsed_time(t1e) / K
    # forward alone, for reference
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.no_grad():
        f0.record(stream)
        for i in range(3):
            mg.lstsq(A0, b0)
        f1.record(stream)
    torch.cuda.synchronize(dev)
    fwd_ms = f0.elapsed_time(f1) / 3
    # end to end: pinned host batch -> device, forward + adjoint, gradients -> host
    Ah = torch.from_numpy(np.stack([h[0] for h in host])).pin_memory()
    bh = torch.from_numpy(np.stack([h[2] for h in host])).pin_memory()
    gAh = torch.empty_like(Ah).pin_memory()
    gbh = torch.empty_like(bh).pin_memory()

    def e2e_step():
        Ad = Ah.to(dev, non_blocking=True).requires_grad_(True)
        bd = bh.to(dev, non_blocking=True).requires_grad_(True)
        x = mg.lstsq(Ad, bd)
        x.backward(gradient=2.0 * x.detach())
        gAh.copy_(Ad.grad, non_blocking=True)
        gbh.copy_(bd.grad, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    Ke = 3
    e0.record(stream)
    for _ in range(Ke):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = e0.elapsed_time(e1) / Ke
    ms, e2e_ms, fwd_ms = max_over_ranks([ms, e2e_ms, fwd_ms], dev, world)
    if rank != 0:
        return 0
    ops = B * fp64_ops(L, m, n)
    peaks = read_peaks()
    peak_ops = peak_fp64_ops_per_s(float(peaks.get("sm_max_mhz", 2070.0)))
    line = {
        "metric": METRIC, "value": world * B / (ms / 1000.0), "unit": "systems/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": diff_config(args.workload, world),
        "through": "torch.autograd.Function (the forward solve and the hand-written adjoint kernel)",
        "e2e": {"value": world * B / (e2e_ms / 1000.0), "unit": "systems/s",
                "h2d_bytes_per_step": Ah.numel() * 8 + bh.numel() * 8,
                "d2h_bytes_per_step": gAh.numel() * 8 + gbh.numel() * 8},
        "gpu_launches": 2 * K,
        "roofline": {"bound": "alu", "achieved": 2 * ops / (ms / 1000.0) / 1e12, "peak": 2 * peak_ops / 1e12,
                     "unit": "TFLOP/s", "frac": ops / (ms / 1000.0) / peak_ops, "traffic": None,
                     "note": "algorithmic FP64 instructions of the forward solves only (%.4g) per step" % ops},
        "forward_only": {"value": world * B / (fwd_ms / 1000.0), "unit": "systems/s", "ms": fwd_ms},
        "backward_overhead": (ms - fwd_ms) / fwd_ms,
    }
    if clk:
        line["clocks"] = clk
    print(json.dumps(line))
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT,
                    choices=sorted(WORKLOADS) + sorted(BATCHED) + sorted(DIFF) + sorted(NEWTON))
    ap.add_argument("--seq-sample", type=int, default=64, help="systems solved one by one for the comparison")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sweep", action="store_true",
                    help="one line per point of the m = n in {64, 128, 256, 512} DD and QD sweep")
    ap.add_argument("--tables", action="store_true",
                    help="one line per size of the paper's Tables 4 and 5, beside its C2050 seconds")
    args = ap.parse_args(argv)
    if args.tables and args.impl == "ours":
        return run_tables(args)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist

        dist.init_process_group("nccl")
    if args.impl == "reference":
        config, unit = workload_config(args.workload, world)
        return run_reference(args, config, unit, rank, world)
    if args.workload in NEWTON:
        return run_gpu_newton(args, rank, world)
    if args.workload in DIFF:
        return run_gpu_diff(args, rank, world)
    if args.workload in BATCHED:
        return run_gpu_batched(args, rank, world)
    if args.sweep:
        args.no_cpu_baseline = True
        for wl in SWEEP:
            args.workload = wl
            L, m, n, extreme = WORKLOADS[wl]
            rc = run_gpu(args, L, m, n, extreme, rank, world)
            if rc:
                return rc
        return 0
    L, m, n, extreme = WORKLOADS[args.workload]
    return run_gpu(args, L, m, n, extreme, rank, world)


if __name__ == "__main__":
    sys.exit(main())
