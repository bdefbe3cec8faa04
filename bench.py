#!/usr/bin/env python
"""Benchmark of the RRS depth hot path on GB300.

Default workload (one "step"): projection depth and asymmetric projection depth
of 1,000 queries uniform in [-4, 4]^10 against X = 10,000 points in d = 10
(95% N(0, I), 5% N(6*1, I)), FP32, k = 1,000 directions over r = 20 rounds,
alpha = 0.7 -- both kinds, every round, every query.  The metric is
query-depths per second (and point-direction projections per second).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``--impl reference`` times the CPU FP64 oracle on the host cores instead (a
bounded sample of the same workload per step).  For N > 1 (torchrun) every
rank runs its own replica of the workload (weak scaling; the path needs no
data exchange) and the slowest rank's time is reported.

Other workloads (``--workload``, one GPU): ``c1`` halfspace depth at d = 2 on FP64
data (launch-bound); ``c3`` halfspace depth at d = 50 on
the tensor cores against the FP32 path; ``c4`` 256 datasets in one batched,
graph-captured launch sequence; ``c5`` continuous-batching serving with p50 /
p99 latency (``--sweep`` for a rate sweep); ``grid`` the paper's per-point
timing grid (its Tables 1 and 2); ``ranks`` its center-outward ranking
correlations at n = 100,000 (Tables 4 and 5); ``convergence`` its
cap-shrinkage study (Sec. 5.1).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "RRS query-depths/sec & point·direction projections/sec; serving p50/p99 latency"
UNIT = "query-depths/s"
WORKLOAD = ("projection + asymmetric projection depth, d=10, n=10000 (95% N(0,I), 5% N(6*1,I)), "
            "1000 queries U[-4,4]^10, k=1000 dirs over r=20 rounds, alpha=0.7, FP32")
SM_COUNT = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ_NOMINAL = 2070.0
# Counters of the dominant kernels from ncu captures of the same launch shapes on a GB300 (profiles/ gives
# the commands): DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch, and for the selection
# kernel its executed warp instructions (smsp__inst_executed.sum) per (point, direction) element.  Each is
# valid only for the kernel source it was taken from: `src_sha16` is the SHA-256 prefix of those files at
# capture time, and a mismatch (the kernel changed since) reports null.
CAPTURED = {
    # k_pdap2<2,12>, d = 10, n = 10,000, 50,000 directions per launch: rounds 10-12 of each kind (six launches
    # of the first warm-up step): DRAM bytes and warp instructions per (point, direction) element, averaged
    "k_pdap2_c2": {"src": ("paper_2506_08262_gb300/csrc/pdap.cu", "paper_2506_08262_gb300/csrc/rrs_internal.h"),
                   "src_sha16": "8f7dbf26a8a98cf6", "traffic": 3.548e6, "warp_instr_per_element": 2.105},
    # k_hd_tc<256>, 10,000 queries x 100 directions x 100,000 points, d = 50: one launch
    "k_hd_tc_c3": {"src": ("paper_2506_08262_gb300/csrc/hd_tc.cu", "paper_2506_08262_gb300/csrc/async_sync.cuh",
                           "paper_2506_08262_gb300/csrc/rrs_device.cuh"),
                   "src_sha16": "78f16dea39c9afd0", "traffic": 290.41e6},
}
ISSUE_PER_SM_PER_CLK = 4     # one warp instruction per clock on each of the four SM sub-partitions


def src_sha16(files) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def captured(key: str, field: str):
    """A captured counter, or None when it was never taken or the kernel source changed since."""
    c = CAPTURED[key]
    if c.get(field) is None or c["src_sha16"] is None or c["src_sha16"] != src_sha16(c["src"]):
        return None
    return c[field]
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-full", action="store_true",
                    help="--impl reference: time the oracle on every query of the workload per step")
    ap.add_argument("--no-autotune", action="store_true",
                    help="headline: keep the shared-memory heuristic for the selection kernel's directions per CTA")
    ap.add_argument("--no-halfspace", action="store_true", help="skip the secondary d=50 halfspace measurement")
    ap.add_argument("--nq", type=int, default=0, help="queries (default: the full workload)")
    ap.add_argument("--workload", choices=["c1", "c2", "c3", "c4", "c5", "grid", "ranks", "convergence"], default="c2",
                    help="c1: halfspace d=2, FP64 data (launch-bound); c2: PD+AP d=10 (the headline); "
                         "c3: halfspace d=50, tensor-core vs FP32 paths; "
                         "c4: 256 datasets batched in one graph-captured launch sequence; c5: serving; "
                         "grid: the paper's projection-depth timing grid (its Tables 1 and 2); "
                         "ranks: its center-outward ranking correlations (Tables 4 and 5); "
                         "convergence: its cap-shrinkage convergence study (Sec. 5.1)")
    ap.add_argument("--scale", type=float, default=1.0, help="c4/c5: shrink n and query counts (tests)")
    ap.add_argument("--sweep", action="store_true", help="c5: serve the stream at 1/8 .. 2x --rate and report each")
    ap.add_argument("--grid-d", type=int, nargs="*", default=None, help="grid: only these dimensions")
    ap.add_argument("--grid-k", type=int, nargs="*", default=None, help="grid: only these direction counts (r = 1)")
    ap.add_argument("--rate", type=float, default=2000.0, help="c5: Poisson arrival rate (requests/s)")
    ap.add_argument("--window", type=float, default=3.0, help="c5: arrival window (s)")
    ap.add_argument("--rates", type=float, nargs="*", default=None, help="c5 --sweep: arrival rates (requests/s)")
    ap.add_argument("--work-limit", type=float, default=None,
                    help="c5: the server's work limit per step (weighted point-direction pairs; 0 = none)")
    return ap.parse_args()


def aggregate_over_ranks(step_ms: float, device=None) -> float:
    """Slowest rank's time (all_reduce MAX); the rank's own time when not distributed."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return step_ms
    t = torch.tensor([step_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: float, world: int, step_ms: float) -> float:
    """Whole-job throughput: every rank processes its own replica of the work (weak scaling)."""
    return world * units_per_rank / (step_ms / 1000.0)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---------------------------------------------------------------------------------------------
# clocks sampling during the timed region
# ---------------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return float("nan")
        sm = np.array([num(r[1]) for r in rows])
        mx = np.array([num(r[2]) for r in rows])
        pw = np.array([num(r[3]) for r in rows])
        load = sm[pw > np.nanmedian(pw) * 0.8] if np.isfinite(pw).any() else sm
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for i, nm in enumerate(names):
                if r[5 + i].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.nanmedian(load if load.size else sm)), "sm_max_mhz": float(np.nanmax(mx)),
                "samples": len(rows), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# ---------------------------------------------------------------------------------------------

def oracle_sample_rate(per_kind: int):
    """Time the FP64 oracle, as it stands, on `per_kind` queries of each kind (all host cores)."""
    import oracle
    oracle.build()
    threads = oracle.max_threads()
    out = {}
    total_q = 0
    t0 = time.perf_counter()
    for kind in (workloads.PROJECTION, workloads.ASYM_PROJECTION):
        Pr = workloads.c2(kind=kind)
        q = np.arange(per_kind)
        oracle.rrs(Pr.X, Pr.Z[q], kind, Pr.k, Pr.r, Pr.alpha, Pr.seed, qidx=q, nthreads=threads)
        total_q += per_kind
    dt = time.perf_counter() - t0
    out["value"] = total_q / dt
    out["seconds"] = dt
    out["cores"] = threads
    out["sample"] = (f"{per_kind} queries of each kind (PD, AP) of the same workload, full n/k/r, "
                     f"OpenMP over queries on {threads} host threads")
    return out


def run_reference(args):
    """The reference arm: the CPU FP64 oracle, as it stands, on the host cores.  Default: a bounded sample
    of the projection-depth workload per step.  --cpu-full: every query of that workload (1,000 of each
    kind) per step.  --workload c3: the d = 50 halfspace workload on its first --nq queries (default 8)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    if args.workload == "c1":
        P = workloads.c1()
        threads = oracle.max_threads()
        times = []
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            oracle.rrs(P.X, P.Z, workloads.HALFSPACE, P.k, P.r, P.alpha, P.seed, nthreads=threads)
            if i >= args.warmup:
                times.append(time.perf_counter() - t0)
        value = P.Z.shape[0] * len(times) / sum(times)
        sample = f"all {P.Z.shape[0]} queries of the d=2 halfspace workload, OpenMP over queries on {threads} host threads"
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "query-depths/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sum(times) / len(times),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": WORKLOAD_C1, "step": sample},
                "cpu_baseline": {"value": value, "unit": "query-depths/s", "cores": threads, "kind": "oracle",
                                 "sample": sample},
                "e2e": {"value": value, "unit": "query-depths/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    if args.workload == "c3":
        P = workloads.c3(nq=args.nq or 8)
        threads = oracle.max_threads()
        times = []
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            oracle.rrs(P.X, P.Z, workloads.HALFSPACE, P.k, P.r, P.alpha, P.seed, nthreads=threads)
            if i >= args.warmup:
                times.append(time.perf_counter() - t0)
        value = P.Z.shape[0] * len(times) / sum(times)
        sample = (f"{P.Z.shape[0]} queries of the d=50 halfspace workload (full n, k, r), OpenMP over queries on "
                  f"{threads} host threads")
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "query-depths/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sum(times) / len(times),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": WORKLOAD_C3, "step": sample},
                "cpu_baseline": {"value": value, "unit": "query-depths/s", "cores": threads, "kind": "oracle",
                                 "sample": sample},
                "e2e": {"value": value, "unit": "query-depths/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    per_kind = 1000 if args.cpu_full else max(1, oracle.max_threads())
    for _ in range(args.warmup):
        oracle_sample_rate(per_kind)
    times = []
    nq = 0
    for _ in range(args.steps):
        r = oracle_sample_rate(per_kind)
        times.append(r["seconds"])
        nq += 2 * per_kind
    value = nq / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sum(times) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "step": f"{per_kind} queries per kind" +
                   (" (the whole workload)" if args.cpu_full else " (bounded sample)")},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                         "sample": r["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------------

def alu_ops_per_element(kind: int, d: int) -> int:
    """Algorithmic ALU operations per (point, direction) element of the selection kernel:
    d FMAs of the projection, 3 per histogram pass of each order-statistic selection
    (bucket index FMA, conversion, shared-memory increment) for the two selections
    (median, then MAD or MAD_+), and 2 for the count of y > med (asymmetric only)."""
    return d + 2 * 3 + (2 if kind == workloads.ASYM_PROJECTION else 0)


def executed_work(captured_shape: bool, elements_per_launch: float, avg_launch_ms: float):
    """The selection kernel's executed instructions (all passes: projection, histograms, gathers, exact
    ranks) against the SM issue peak, for the launch shape whose instruction count was measured on the
    current kernel source (else None)."""
    wipe = captured("k_pdap2_c2", "warp_instr_per_element")
    if not captured_shape or wipe is None:
        return None
    instr_per_s = elements_per_launch * wipe / (avg_launch_ms / 1000)
    peak = SM_COUNT * ISSUE_PER_SM_PER_CLK * SM_MAX_MHZ_NOMINAL * 1e6
    return {"warp_instr_per_element": wipe, "achieved_warp_instr_per_s": instr_per_s,
            "peak_warp_instr_per_s": peak, "frac": instr_per_s / peak,
            "source": "instructions per element from ncu smsp__inst_executed.sum; issue peak 152 SMs x 4 x 2070 MHz"}


def run_ours(args):
    import torch
    import torch.distributed as dist

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from __graft_entry__ import build
    if rank == 0 or world == 1:
        build()
    if world > 1:
        dist.barrier()
    import paper_2506_08262_gb300 as rrs

    kinds = (workloads.PROJECTION, workloads.ASYM_PROJECTION)
    P2 = workloads.c2()
    # every rank holds the data cloud and takes its own queries of the workload's law (rank 0 the workload's
    # own), so per-GPU work is fixed and no data is exchanged
    X, Z = P2.X, workloads.c2_queries(rank, args.nq or P2.nq)
    nq, n, d = Z.shape[0], X.shape[0], X.shape[1]
    k, r, alpha, seed = P2.k, P2.r, P2.alpha, P2.seed
    m = -(-k // r)

    ctx = rrs.rrs_create(local, 0)
    Xd = torch.from_numpy(X).to(dev)
    did = rrs.rrs_register_dataset(ctx, Xd, n, d, rrs.RRS_F32, True)
    Zd = torch.from_numpy(Z).to(dev)
    outs = {kd: torch.empty(nq, dtype=torch.float64, device=dev) for kd in kinds}
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    # the autotuner times each choice; --no-autotune keeps the library's shared-memory heuristic (used for
    # profiler captures, where the probe timings are distorted by the profiler itself)
    tuned = ({workloads.KIND_NAMES[kd]: rrs.rrs_autotune(ctx, did, kd, k, r) for kd in kinds}
             if not args.no_autotune else "heuristic")

    def step():
        for kd in kinds:
            rrs.rrs_depth(ctx, did, Zd, nq, rrs.RRS_F32, True, kd, k, r, alpha, seed, rrs.RRS_PREC_FP32_SIMT,
                          outs[kd], None, None, None, True, stream)

    for _ in range(max(3, args.warmup)):
        step()
    rrs.rrs_check(ctx, stream)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = rrs.rrs_launch_count(ctx)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()                     # L2 flush between timed steps (not timed)
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    launches = rrs.rrs_launch_count(ctx) - launches0
    rrs.rrs_check(ctx, stream)
    step_ms = aggregate_over_ranks(float(sum(a.elapsed_time(b) for a, b in ev)) / args.steps, dev)
    # per-kernel device times from a second pass over the same K steps with the library's per-launch CUDA
    # events (recorded on the launching stream); the headline above ran without them
    rrs.rrs_profile_enable(ctx, True)
    for _ in range(args.steps):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    prof = rrs.rrs_profile_read(ctx)
    rrs.rrs_profile_enable(ctx, False)
    rrs.rrs_check(ctx, stream)
    clocks = sampler.stop()

    # end to end through the public API: pinned host query buffer in, host depths out
    Zh = torch.from_numpy(Z).pin_memory()
    outh = {kd: torch.empty(nq, dtype=torch.float64).pin_memory() for kd in kinds}

    def step_e2e():
        for kd in kinds:
            rrs.rrs_depth(ctx, did, Zh, nq, rrs.RRS_F32, False, kd, k, r, alpha, seed, rrs.RRS_PREC_FP32_SIMT,
                          outh[kd], None, None, None, False, stream)

    step_e2e()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e2e_times = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step_e2e()
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
    e2e_ms = aggregate_over_ranks(1000 * float(np.mean(e2e_times)), dev)
    for kd in kinds:
        assert np.array_equal(outh[kd].numpy(), outs[kd].cpu().numpy()), "e2e results differ from device results"

    qd_per_step = len(kinds) * nq
    value = job_value(qd_per_step, world, step_ms)
    pd_per_step = len(kinds) * nq * r * m * n

    # roofline of the dominant kernel (selection kernel, plain ALU bound)
    pd_ms, pd_launches = prof["pdap"]
    ops_per_step = sum(nq * r * m * n * alu_ops_per_element(kd, d) for kd in kinds)
    launches_per_step = max(1, pd_launches // args.steps)
    ops_per_launch = ops_per_step / launches_per_step
    avg_launch_ms = pd_ms / max(1, pd_launches)
    achieved = ops_per_launch / (avg_launch_ms / 1000) / 1e9
    peak = SM_COUNT * FP32_LANES_PER_SM * SM_MAX_MHZ_NOMINAL * 1e6 / 1e9
    stage_share = {k2: round(v[0] / max(1e-9, sum(x[0] for x in prof.values())), 4) for k2, v in prof.items()
                   if v[1]}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "global_batch": qd_per_step * world, "queries_per_kind": nq,
                   "n": n, "d": d, "k": k, "r": r, "alpha": alpha,
                   "parallelism": f"query shards over {world} GPU(s), data cloud replicated, no collective on the data path",
                   "l2": "flushed between timed steps (512 MiB device write); inputs smaller than L2",
                   "autotuned_directions_per_cta": tuned},
        "pd_per_s": world * pd_per_step / (step_ms / 1000),
        "gpu_launches": int(launches),
        "e2e": {"value": job_value(qd_per_step, world, e2e_ms), "unit": UNIT,
                "h2d_bytes_per_step": int(Zh.numel() * 4 * len(kinds)),
                "d2h_bytes_per_step": int(nq * 8 * len(kinds))},
        "roofline": {"bound": "alu", "kernel": "k_pdap", "achieved": achieved, "peak": peak, "unit": "Gop/s",
                     "frac": achieved / peak, "traffic": captured("k_pdap2_c2", "traffic") if args.nq == 0 else None,
                     "peak_source": "152 SMs x 128 FP32/INT32 lanes x 2070 MHz (recipe unit counts and max clock)",
                     "ops_per_launch": ops_per_launch, "avg_launch_ms": avg_launch_ms,
                     "executed": executed_work(args.nq == 0, nq * r * m * n * len(kinds) / launches_per_step,
                                               avg_launch_ms)},
        "stage_ms_per_step": {k2: v[0] / args.steps for k2, v in prof.items() if v[1]},
        "stage_share": stage_share,
        "kernel_timing": "stage and kernel times from a second pass over the same K steps with per-launch CUDA "
                         "events on the launching stream; the headline value from a pass without them",
        "clocks": clocks,
        "wall_s_timed": wall,
    }
    if rank == 0 and world == 1 and not args.no_halfspace:
        # secondary: the tensor-core halfspace path on the full d=50 workload (10,000 queries) against the
        # FP32 path on its first 1,000 queries
        line["halfspace_d50"] = measure_halfspace(10_000, 2, 3, nq_fp32=1000)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = oracle_sample_rate(5 * max(1, os.cpu_count() or 1))
        line["cpu_baseline"] = {"value": cb["value"], "unit": UNIT, "cores": cb["cores"], "kind": "oracle",
                                "sample": cb["sample"]}
    rrs.rrs_free(ctx, did)
    rrs.rrs_destroy(ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


WORKLOAD_C1 = ("halfspace depth, d=2, n=1000 N(0,I) rows, 100 queries N(0,1.5^2 I), k=1000 dirs over r=10 rounds, "
               "alpha=0.5, FP64 data")


def run_c1(args):
    """Halfspace depth at d=2 on FP64 data: 100 queries of 1,000 directions over 10 rounds, through rrs_depth
    (FP32 path with the exact FP64 re-check).  The whole call is a few small launches per round, so it is
    launch-bound and no roofline is claimed; the line reports the call's time and its launches."""
    import torch
    from __graft_entry__ import build
    build()
    import paper_2506_08262_gb300 as rrs
    dev = torch.device("cuda", 0)
    P = workloads.c1()
    ctx = rrs.rrs_create(0, 0)
    did = rrs.rrs_register_dataset(ctx, torch.from_numpy(P.X).to(dev), P.X.shape[0], 2, rrs.RRS_F64, True)
    Zd = torch.from_numpy(P.Z).to(dev)
    nq = P.Z.shape[0]
    dep = torch.empty(nq, dtype=torch.float64, device=dev)
    cnt = torch.empty(nq, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        rrs.rrs_depth(ctx, did, Zd, nq, rrs.RRS_F64, True, rrs.RRS_HALFSPACE, P.k, P.r, P.alpha, P.seed,
                      rrs.RRS_PREC_FP32_SIMT, dep, cnt, None, None, True, stream)
    for _ in range(max(3, args.warmup)):
        step()
    rrs.rrs_check(ctx, stream)
    torch.cuda.synchronize()
    launches0 = rrs.rrs_launch_count(ctx)
    evs = []
    for _ in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    launches = (rrs.rrs_launch_count(ctx) - launches0) // args.steps
    rrs.rrs_check(ctx, stream)
    rrs.rrs_free(ctx, did)
    rrs.rrs_destroy(ctx)
    line = {"metric": METRIC, "value": nq / (ms / 1000), "unit": "query-depths/s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 projections, f64 data and exact re-check", "data": "synthetic",
            "config": {"workload": WORKLOAD_C1, "l2": "inputs far smaller than L2; launch-bound"},
            "gpu_launches_per_step": int(launches), "roofline": None}
    print(json.dumps(line), flush=True)


WORKLOAD_C3 = ("halfspace depth, d=50, n=100000 Student-t(3) rows mapped by a random SPD square root, "
               "10000 queries from the same law, k=2000 dirs over r=20 rounds, alpha=0.9, FP32 data")


def measure_halfspace(nq: int, steps: int, warmup: int, nq_fp32: int = 0):
    """Halfspace depth at d=50: split-BF16x3 tensor-core path on `nq` queries of the d=50 workload (full n,
    k, r) against the FP32 CUDA-core path on the first `nq_fp32` of them (default all).  A query's result does
    not depend on the batch, so the counts are compared on the common queries.  Returns a dict with both
    arms and the speedup in query-depths per second."""
    import torch
    import paper_2506_08262_gb300 as rrs
    dev = torch.device("cuda", 0)
    P = workloads.c3(nq=nq)
    n, d, k, r = P.n, P.d, P.k, P.r
    m = -(-k // r)
    ctx = rrs.rrs_create(0, 0)
    did = rrs.rrs_register_dataset(ctx, torch.from_numpy(P.X).to(dev), n, d, rrs.RRS_F32, True)
    Zd = torch.from_numpy(P.Z).to(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    bf16_peak = float(peaks.get("bf16_tflops_sustained", 1700.0))
    out, results = {}, {}
    nq_arm = {"tc": nq, "fp32": nq_fp32 or nq}
    for name, prec in (("tc", rrs.RRS_PREC_SPLIT_BF16X3), ("fp32", rrs.RRS_PREC_FP32_SIMT)):
        na = nq_arm[name]
        dep = torch.empty(na, dtype=torch.float64, device=dev)
        cnt = torch.empty(na, dtype=torch.int64, device=dev)

        def step():
            rrs.rrs_depth(ctx, did, Zd, na, rrs.RRS_F32, True, rrs.RRS_HALFSPACE, k, r, P.alpha, P.seed, prec,
                          dep, cnt, None, None, True, stream)
        for _ in range(max(3, warmup)):
            step()
        rrs.rrs_check(ctx, stream)
        torch.cuda.synchronize()
        sampler = ClockSampler(0)
        sampler.start()
        rrs.rrs_profile_enable(ctx, True)
        evs = []
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step()
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        prof = rrs.rrs_profile_read(ctx)
        rrs.rrs_profile_enable(ctx, False)
        clocks = sampler.stop()
        rrs.rrs_check(ctx, stream)
        ms = sum(a.elapsed_time(b) for a, b in evs) / steps
        stage = "hd_tc" if prec == rrs.RRS_PREC_SPLIT_BF16X3 else "hd_simt"
        kms, kl = prof[stage]
        elems_per_launch = na * m * n
        avg_ms = kms / max(1, kl)
        entry = {"queries": na, "ms_per_step": ms, "value": na / (ms / 1000), "unit": "query-depths/s",
                 "pd_per_s": na * r * m * n / (ms / 1000), "kernel_ms_per_launch": avg_ms,
                 "kernel_share": kms / max(1e-9, sum(v[0] for v in prof.values())), "clocks": clocks}
        if name == "tc":
            flops = 6.0 * d * elems_per_launch   # three BF16 products of d terms per point-direction pair
            achieved = flops / (avg_ms / 1000) / 1e12
            entry["roofline"] = {"bound": "tensor", "kernel": "k_hd_tc", "achieved": achieved, "peak": bf16_peak,
                                 "unit": "TFLOP/s", "frac": achieved / bf16_peak,
                                 "traffic": captured("k_hd_tc_c3", "traffic") if nq == 10_000 else None,
                                 "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (of measured)",
                                 "flops_per_launch": flops}
        else:
            flops = 2.0 * d * elems_per_launch
            peak = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12
            achieved = flops / (avg_ms / 1000) / 1e12
            entry["roofline"] = {"bound": "alu", "kernel": "k_hd_simt", "achieved": achieved, "peak": peak,
                                 "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                                 "peak_source": "152 SMs x 128 FP32 FMA lanes x 2 x 2070 MHz"}
        results[name] = cnt.cpu().numpy()
        out[name] = entry
    common = min(nq_arm.values())
    same = bool(np.array_equal(results["tc"][:common], results["fp32"][:common]))
    # near-tie re-check rate of the tensor-core epilogue: the round-1 directions of a sample of queries,
    # counted by the debug entry point (points whose fast sign was not trusted / all point-direction pairs)
    ns = min(nq, 16)
    U = torch.empty((ns, m, d), dtype=torch.float32, device=dev)
    for q in range(ns):
        rrs.rrs_debug_directions(ctx, P.seed, q, 1, m, d, P.alpha, None, U[q])
    band = torch.zeros(ns, dtype=torch.int64, device=dev)
    dep = torch.empty((ns, m), dtype=torch.float64, device=dev)
    rrs.rrs_debug_round_depths(ctx, did, Zd[:ns].contiguous(), ns, rrs.RRS_F32, rrs.RRS_HALFSPACE, m, U,
                               rrs.RRS_PREC_SPLIT_BF16X3, dep, None, band)
    torch.cuda.synchronize()
    recheck = {"rate": float(band.sum().item()) / (ns * m * n), "sample": f"{ns} queries x {m} round-1 directions x n",
               "rechecks": int(band.sum().item())}
    rrs.rrs_free(ctx, did)
    rrs.rrs_destroy(ctx)
    return {"workload": WORKLOAD_C3, "queries": nq, "n": n, "d": d, "k": k, "r": r, "tensor_core": out["tc"],
            "fp32_cuda_core": out["fp32"], "speedup_tc_over_fp32": out["tc"]["value"] / out["fp32"]["value"],
            "counts_identical": same, "counts_compared_on_queries": common, "tensor_core_recheck": recheck}


def run_c3(args):
    """Halfspace depth at d=50: split-BF16x3 tensor-core path against the FP32 CUDA-core path."""
    from __graft_entry__ import build
    build()
    h = measure_halfspace(args.nq or 10_000, args.steps, args.warmup, nq_fp32=min(args.nq or 10_000, 1000))
    line = {"metric": METRIC, "value": h["tensor_core"]["value"], "unit": "query-depths/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": h["tensor_core"]["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3->f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_C3, "n": h["n"], "d": h["d"], "queries": h["queries"], "k": h["k"],
                       "r": h["r"], "l2": "flushed between timed steps (512 MiB device write)"},
            **{key: h[key] for key in ("tensor_core", "fp32_cuda_core", "speedup_tc_over_fp32", "counts_identical",
                                       "tensor_core_recheck")}}
    assert h["counts_identical"], "tensor-core and FP32 counts differ"
    print(json.dumps(line), flush=True)


def roofline_mix(prof, problems, bf16_peak):
    """Per-stage rooflines of one profiled batched call and their time-weighted mix: each stage's algorithmic
    work over the requests that reach it, divided by the stage's device time, against that stage's peak."""
    fp32 = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12      # TFLOP/s (FMA = 2)
    alu = SM_COUNT * FP32_LANES_PER_SM * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12           # T ops/s
    work = {"hd_tc": 0.0, "hd_simt": 0.0, "keys": 0.0, "pdap": 0.0}
    for P in problems:
        pairs = float(P.nq) * P.r * P.m * P.n
        if P.kind == workloads.HALFSPACE:
            if P.d + 2 <= 128:
                work["hd_tc"] += 6.0 * P.d * pairs
            else:
                work["hd_simt"] += 2.0 * P.d * pairs
        else:
            keys = P.d > 16 or P.n > 55_000   # keys formed by their own kernel
            if keys:
                work["keys"] += 2.0 * P.d * pairs
            work["pdap"] += (alu_ops_per_element(P.kind, P.d) - (P.d if keys else 0)) * pairs
    peaks = {"hd_tc": (bf16_peak, "TFLOP/s"), "hd_simt": (fp32, "TFLOP/s"), "keys": (fp32, "TFLOP/s"),
             "pdap": (alu, "Top/s")}
    stages, num, den = {}, 0.0, 0.0
    for name, w in work.items():
        ms = prof.get(name, (0.0, 0))[0]
        if w <= 0 or ms <= 0:
            continue
        achieved = w / (ms / 1000) / 1e12
        peak, unit = peaks[name]
        stages[name] = {"ms": ms, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak}
        num += achieved / peak * ms
        den += ms
    other = sum(v[0] for k, v in prof.items() if k not in stages)
    return {"stages": stages, "time_weighted_frac": num / den if den else None, "other_stages_ms": other,
            "how": "one profiled batched call (no graph); algorithmic work per stage / stage device time; "
                   "halfspace 6d FLOP per pair against the sustained BF16 peak, keys 2d FLOP per pair against "
                   "the FP32 FMA peak, selection d+6 (+2 for D_AP; without the d projection FMAs when keys come "
                   "from the keys kernel) ops per pair against the ALU peak"}


WORKLOAD_C4 = ("batched: 256 datasets, n log-uniform [500, 50000], d uniform {5..100}, N(mu_k, Sigma_k), "
               "1..1000 queries each, kind uniform over halfspace/projection/asymmetric, k=1000 over r=10, "
               "alpha=0.9, FP32")


def run_c4(args):
    """All requests of the batched workload in one graph-captured launch sequence, against the same
    requests issued one rrs_depth call at a time."""
    import torch
    from __graft_entry__ import build
    build()
    import paper_2506_08262_gb300 as rrs
    dev = torch.device("cuda", 0)
    problems = workloads.c4(scale=args.scale)
    ctx = rrs.rrs_create(0, 0)
    stream = torch.cuda.current_stream(dev)
    reqs, keep = [], []
    total_q = 0
    pd_total = 0
    for i, P in enumerate(problems):
        did = rrs.rrs_register_dataset(ctx, torch.from_numpy(P.X).to(dev), P.n, P.d, rrs.RRS_F32, True)
        Z = torch.from_numpy(P.Z).to(dev)
        out = torch.empty(P.nq, dtype=torch.float64, device=dev)
        keep.append((did, Z, out, P))
        reqs.append(rrs.rrs_request(dataset_id=did, Z=Z.data_ptr(), n_queries=P.nq, dtype=rrs.RRS_F32,
                                    kind=P.kind, n_dirs=P.k, n_refinements=P.r, cap_shrink=P.alpha, seed=P.seed,
                                    depth_out=out.data_ptr()))
        total_q += P.nq
        pd_total += P.nq * P.r * (-(-P.k // P.r)) * P.n
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def timed(fn, steps):
        evs = []
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs) / steps

    # the same requests with halfspace depth on the tensor cores (split-BF16x3; exact counts)
    reqs_tc = []
    for q in reqs:
        c = rrs.rrs_request()
        ctypes.pointer(c)[0] = q
        if c.kind == rrs.RRS_HALFSPACE and keep[len(reqs_tc)][3].d + 2 <= 128:
            c.precision = rrs.RRS_PREC_SPLIT_BF16X3
        reqs_tc.append(c)

    def batched():
        rrs.rrs_depth_batched(ctx, reqs_tc, use_graph=True, stream=stream)

    def batched_fp32():
        rrs.rrs_depth_batched(ctx, reqs, use_graph=True, stream=stream)

    def one_by_one():
        for did, Z, out, P in keep:
            rrs.rrs_depth(ctx, did, Z, P.nq, rrs.RRS_F32, True, P.kind, P.k, P.r, P.alpha, P.seed,
                          rrs.RRS_PREC_FP32_SIMT, out, None, None, None, True, stream)

    for _ in range(max(3, args.warmup)):
        batched()
    rrs.rrs_check(ctx, stream)
    sampler = ClockSampler(0)
    sampler.start()
    launches0 = rrs.rrs_launch_count(ctx)
    ms_b = timed(batched, args.steps)
    launches = rrs.rrs_launch_count(ctx) - launches0
    clocks = sampler.stop()
    res_b = [out.cpu().numpy().copy() for _, _, out, _ in keep]
    for _ in range(2):
        batched_fp32()
    ms_f = timed(batched_fp32, args.steps)
    res_f = [out.cpu().numpy().copy() for _, _, out, _ in keep]
    one_by_one()
    torch.cuda.synchronize()
    ms_s = timed(one_by_one, max(1, args.steps // 2))
    rrs.rrs_check(ctx, stream)
    same = all(np.array_equal(res_b[i], keep[i][2].cpu().numpy()) and np.array_equal(res_f[i], res_b[i])
               for i in range(len(keep)))
    line = {"metric": METRIC, "value": total_q / (ms_b / 1000), "unit": "query-depths/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms_b, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3->f32 (halfspace), f32 (projection)",
            "data": "synthetic",
            "config": {"workload": WORKLOAD_C4, "datasets": len(problems), "queries": total_q, "scale": args.scale,
                       "l2": "flushed between timed steps (512 MiB device write)"},
            "pd_per_s": pd_total / (ms_b / 1000), "gpu_launches": int(launches),
            "batched_fp32": {"ms_per_step": ms_f, "value": total_q / (ms_f / 1000)},
            "one_call_per_request_fp32": {"ms_per_step": ms_s, "value": total_q / (ms_s / 1000)},
            "speedup_batched_over_per_request": ms_s / ms_b, "speedup_tensor_cores_in_batch": ms_f / ms_b,
            "results_identical": bool(same), "clocks": clocks}
    # per-stage rooflines of the tensor-core batch (one extra call, timed by the library's stage profiler)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    rrs.rrs_profile_enable(ctx, True)
    rrs.rrs_depth_batched(ctx, reqs_tc, use_graph=False, stream=stream)
    torch.cuda.synchronize()
    prof = rrs.rrs_profile_read(ctx)
    rrs.rrs_profile_enable(ctx, False)
    rrs.rrs_check(ctx, stream)
    line["roofline_mix"] = roofline_mix(prof, problems, float(peaks.get("bf16_tflops_sustained", 1700.0)))
    for did, _, _, _ in keep:
        rrs.rrs_free(ctx, did)
    rrs.rrs_destroy(ctx)
    print(json.dumps(line), flush=True)


WORKLOAD_C5 = ("serving: 64 resident datasets as in the batched workload, Poisson arrivals, 1..4096 queries per "
               "request (log-uniform), kinds 50/30/20 halfspace/projection/asymmetric, k=1000 over r=10, FP32")


def _latency_stats(lat):
    lat = np.sort(np.asarray(lat))
    if lat.size == 0:
        return {"p50_ms": None, "p99_ms": None, "mean_ms": None}
    return {"p50_ms": 1000 * float(np.percentile(lat, 50)), "p99_ms": 1000 * float(np.percentile(lat, 99)),
            "mean_ms": 1000 * float(lat.mean())}


def run_c5(args):
    """Poisson request stream through the continuous-batching server, against one rrs_depth call per
    request in arrival order.  Requests that would push the backlog of waiting queries beyond a bound are
    shed (counted) in both arms.  With --sweep both arms serve the stream at every rate of --rates (default:
    1/8 .. 2x --rate)."""
    import collections
    import torch
    from __graft_entry__ import build
    build()
    import paper_2506_08262_gb300 as rrs
    dev = torch.device("cuda", 0)
    datasets, reqs = workloads.c5(rate=args.rate, window_s=args.window, scale=args.scale)
    ctx = rrs.rrs_create(0, 0)
    stream = torch.cuda.current_stream(dev)
    ids = [rrs.rrs_register_dataset(ctx, torch.from_numpy(X).to(dev), X.shape[0], X.shape[1], rrs.RRS_F32, True)
           for X in datasets]
    k, r, alpha = 1000, 10, 0.9
    max_slots = 16384
    backlog_limit = 2 * max_slots

    # halfspace requests are served on the tensor cores (split-BF16x3, exact counts); the
    # per-request arm is the plain FP32 path
    tc = rrs.RRS_PREC_SPLIT_BF16X3
    # warm the kernels (and build every dataset's BF16 planes before the clock starts)
    w = rrs.rrs_server_create(ctx, 256, 100, 100, stream, precision=tc)
    wids = []
    for kind in (0, 1, 2):
        for di in range(len(ids)):
            if kind and di:
                break
            Zw = np.ascontiguousarray(datasets[di][:2])
            wids.append(rrs.rrs_server_submit(w, ids[di], Zw, 2, rrs.RRS_F32, kind, k, r, alpha, 0, np.zeros(2)))
    while not all(rrs.rrs_server_poll(w, rid) for rid in wids):
        rrs.rrs_server_step(w)
    rrs.rrs_server_destroy(w)
    torch.cuda.synchronize()

    # ---- continuous batching ----------------------------------------------------------------
    def serve_stream(reqs):
        srv = rrs.rrs_server_create(ctx, max_slots, 100, 100, stream, precision=tc)
        if args.work_limit is not None:
            rrs.rrs_server_set_work_limit(srv, args.work_limit)
        outs, lat, shed, served_q, steps = {}, [], 0, 0, 0
        inflight = collections.deque()
        backlog = 0
        t0 = time.perf_counter()
        i = 0
        while i < len(reqs) or outs:
            now = time.perf_counter() - t0
            while i < len(reqs) and reqs[i].t_arrival <= now:
                q = reqs[i]
                nq = q.Z.shape[0]
                if backlog + nq > backlog_limit:
                    shed += 1
                else:
                    out = np.empty(nq)
                    rid = rrs.rrs_server_submit(srv, ids[q.dataset], q.Z, nq, rrs.RRS_F32, q.kind, k, r, alpha, i,
                                                out)
                    outs[rid] = (q.t_arrival, nq, out)
                    backlog += nq
                i += 1
            if outs:
                rrs.rrs_server_step(srv)
                steps += 1
                ev = torch.cuda.Event()
                ev.record(stream)
                inflight.append(ev)
                if len(inflight) > 2:
                    inflight.popleft().synchronize()
            elif i < len(reqs):
                time.sleep(max(0.0, min(0.001, reqs[i].t_arrival - now)))
            for rid in list(outs):
                if rrs.rrs_server_poll(srv, rid):
                    ta, nq, _ = outs.pop(rid)
                    lat.append(time.perf_counter() - t0 - ta)
                    backlog -= nq
                    served_q += nq
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        rrs.rrs_server_destroy(srv)
        rrs.rrs_check(ctx, stream)
        return {"served_requests": len(lat), "shed_requests": shed, "queries": served_q,
                "value": served_q / wall, "wall_s": wall, "steps": steps, **_latency_stats(lat)}

    # ---- one rrs_depth call per request, arrival order ------------------------------------------
    def per_request(reqs):
        lat2, shed2, served2 = [], 0, 0
        queue = collections.deque()
        t0 = time.perf_counter()
        i = 0
        backlog = 0
        while i < len(reqs) or queue:
            now = time.perf_counter() - t0
            while i < len(reqs) and reqs[i].t_arrival <= now:
                nq = reqs[i].Z.shape[0]
                if backlog + nq > backlog_limit:
                    shed2 += 1
                else:
                    queue.append(i)
                    backlog += nq
                i += 1
            if not queue:
                time.sleep(max(0.0, min(0.001, reqs[i].t_arrival - now)) if i < len(reqs) else 0)
                continue
            j = queue.popleft()
            q = reqs[j]
            nq = q.Z.shape[0]
            out = np.empty(nq)
            rrs.rrs_depth(ctx, ids[q.dataset], q.Z, nq, rrs.RRS_F32, False, q.kind, k, r, alpha, j,
                          rrs.RRS_PREC_FP32_SIMT, out, None, None, None, False, stream)
            lat2.append(time.perf_counter() - t0 - q.t_arrival)
            backlog -= nq
            served2 += nq
        wall2 = time.perf_counter() - t0
        return {"served_requests": len(lat2), "shed_requests": shed2, "queries": served2, "value": served2 / wall2,
                "wall_s": wall2, **_latency_stats(lat2)}

    limit_used = args.work_limit if args.work_limit is not None else "library default (RRS_SERVER_DEFAULT_WORK)"
    if args.sweep:
        # both arms at every rate on the same resident datasets; a rate is stable when nothing is shed and
        # the p99 stays below half the arrival window (the backlog does not grow over the window)
        sampler = ClockSampler(0)
        sampler.start()
        sweep = []
        rates = args.rates if args.rates else [args.rate * f for f in (0.125, 0.25, 0.5, 1.0, 2.0)]
        for rate in rates:
            _, rq = workloads.c5(rate=rate, window_s=args.window, scale=args.scale)
            cb = serve_stream(rq)
            pr = per_request(rq)
            sweep.append({"rate_req_per_s": rate, "offered_requests": len(rq),
                          "offered_queries": int(sum(x.Z.shape[0] for x in rq)),
                          "continuous_batching": cb, "one_call_per_request_fp32": pr})
        clocks = sampler.stop()

        def stable(x):
            return x["shed_requests"] == 0 and x.get("p99_ms", 1e30) <= 500.0 * args.window
        for did in ids:
            rrs.rrs_free(ctx, did)
        rrs.rrs_destroy(ctx)
        line = {"metric": METRIC, "value": max(x["continuous_batching"]["value"] for x in sweep),
                "unit": "query-depths/s", "n_gpus": 1, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16x3->f32 (halfspace), f32 (projection)", "data": "synthetic",
                "config": {"workload": WORKLOAD_C5, "window_s": args.window, "scale": args.scale, "slots": max_slots,
                           "backlog_limit_queries": backlog_limit, "work_limit": limit_used,
                           "rates": [x["rate_req_per_s"] for x in sweep]},
                "sweep": sweep,
                "max_stable_rate_req_per_s": {
                    "continuous_batching": max([x["rate_req_per_s"] for x in sweep
                                                if stable(x["continuous_batching"])], default=None),
                    "one_call_per_request_fp32": max([x["rate_req_per_s"] for x in sweep
                                                      if stable(x["one_call_per_request_fp32"])], default=None)},
                "clocks": clocks}
        print(json.dumps(line), flush=True)
        return

    sampler = ClockSampler(0)
    sampler.start()
    cb = serve_stream(reqs)
    clocks = sampler.stop()
    wall = cb["wall_s"]
    pr = per_request(reqs)
    for did in ids:
        rrs.rrs_free(ctx, did)
    rrs.rrs_destroy(ctx)
    line = {"metric": METRIC, "value": cb["value"], "unit": "query-depths/s", "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": 1000 * wall, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x3->f32 (halfspace), f32 (projection)", "data": "synthetic",
            "config": {"workload": WORKLOAD_C5, "rate_req_per_s": args.rate, "window_s": args.window,
                       "requests_offered": len(reqs), "queries_offered": int(sum(x.Z.shape[0] for x in reqs)),
                       "scale": args.scale, "slots": max_slots, "backlog_limit_queries": backlog_limit,
                       "work_limit": limit_used},
            "continuous_batching": cb, "one_call_per_request_fp32": pr, "clocks": clocks}
    print(json.dumps(line), flush=True)


# The paper's per-point projection-depth times in seconds (RTX 4080): Table 1 (n = 10,000, r = 1) and
# Table 2 (n = 10,000, k = 250,000), columns d = 5, 10, 25, 50, 75, 100, 125, 150.
PAPER_GRID_D = (5, 10, 25, 50, 75, 100, 125, 150)
PAPER_TABLE1 = {
    1_000: (0.01,) * 8, 2_500: (0.01,) * 8, 5_000: (0.02,) * 8, 10_000: (0.03,) * 8,
    25_000: (0.06, 0.07, 0.07, 0.07, 0.07, 0.07, 0.07, 0.08),
    50_000: (0.13, 0.14, 0.14, 0.14, 0.14, 0.15, 0.15, 0.16),
    100_000: (0.26, 0.28, 0.28, 0.30, 0.28, 0.28, 0.30, 0.30),
    250_000: (2.49, 2.49, 2.52, 2.59, 2.60, 2.60, 2.64, 2.66),
}
PAPER_TABLE2 = {  # k = 250,000; key = refinements r
    10: (0.62, 0.67, 0.67, 0.69, 0.69, 0.69, 0.74, 0.76),
    25: (0.61, 0.65, 0.65, 0.68, 0.69, 0.69, 0.70, 0.71),
    50: (0.61, 0.65, 0.65, 0.67, 0.68, 0.68, 0.70, 0.73),
    100: (0.66, 0.67, 0.67, 0.68, 0.70, 0.69, 0.71, 0.72),
}


def run_grid(args):
    """Projection depth on the paper's timing grid: n = 10,000 Gaussian points with Toeplitz covariance
    (the paper's generator), one query point at a time (latency) and 32 points per call (time per point),
    every k of Table 1 at r = 1 and every r of Table 2 at k = 250,000, for d = 5 ... 150."""
    import torch
    from __graft_entry__ import build
    build()
    import paper_2506_08262_gb300 as rrs
    dev = torch.device("cuda", 0)
    ctx = rrs.rrs_create(0, 0)
    stream = torch.cuda.current_stream(dev)
    n, batch = 10_000, 32
    rows = []
    sampler = ClockSampler(0)
    sampler.start()

    def time_call(did, Z, nq, k, r, reps):
        dep = torch.empty(nq, dtype=torch.float64, device=dev)
        fn = lambda: rrs.rrs_depth(ctx, did, Z, nq, rrs.RRS_F32, True, rrs.RRS_PROJECTION, k, r, 0.9, 0,
                                   rrs.RRS_PREC_FP32_SIMT, dep, None, None, None, True, stream)
        fn()
        torch.cuda.synchronize()
        evs = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        return min(x.elapsed_time(y) for x, y in evs)

    for di, d in enumerate(PAPER_GRID_D):
        if args.grid_d and d not in args.grid_d:
            continue
        X, Z = workloads.toeplitz_gaussian(1000 + d, n, d, batch)
        did = rrs.rrs_register_dataset(ctx, torch.from_numpy(X).to(dev), n, d, rrs.RRS_F32, True)
        Zd = torch.from_numpy(Z).to(dev)
        cells = [(k, 1, PAPER_TABLE1[k][di]) for k in sorted(PAPER_TABLE1)]
        cells += [(250_000, r, PAPER_TABLE2[r][di]) for r in sorted(PAPER_TABLE2)]
        if args.grid_k:
            cells = [c for c in cells if c[0] in args.grid_k and c[1] == 1]
        for k, r, paper_s in cells:
            reps = 2 if k >= 250_000 else (3 if k >= 100_000 else 5)
            nb = 8 if k >= 250_000 else batch   # bounded run time: 8 points per call at k = 250,000
            one = time_call(did, Zd, 1, k, r, reps)
            many = time_call(did, Zd, nb, k, r, reps) / nb
            rows.append({"d": d, "k": k, "r": r, "paper_s_per_point": paper_s, "ms_one_point": round(one, 4),
                         "batch": nb, "ms_per_point_batched": round(many, 4),
                         "speedup_one_point": round(paper_s * 1000 / one, 1),
                         "speedup_batched": round(paper_s * 1000 / many, 1)})
        rrs.rrs_free(ctx, did)
    clocks = sampler.stop()
    rrs.rrs_check(ctx, stream)
    rrs.rrs_destroy(ctx)
    sp1 = [r_["speedup_one_point"] for r_ in rows]
    spb = [r_["speedup_batched"] for r_ in rows]
    line = {"metric": "projection depth time per query point (paper's timing grid)", "value": None,
            "unit": "ms", "n_gpus": 1, "higher_is_better": False, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "paper timing grid: D_P, n = 10,000 N(0, Toeplitz 2^-|i-j|), d in 5..150, "
                                   "r = 1 with k = 1,000..250,000, and k = 250,000 with r = 10..100",
                       "batch": "32 points per call (8 at k = 250,000)",
                       "timing": "CUDA events around rrs_depth, best of 2-5 after one warm-up"},
            "speedup_vs_paper_one_point": {"min": min(sp1), "median": float(np.median(sp1)), "max": max(sp1)},
            "speedup_vs_paper_batched": {"min": min(spb), "median": float(np.median(spb)), "max": max(spb)},
            "paper_hardware": "RTX 4080 laptop GPU (context only)", "rows": rows, "clocks": clocks}
    print(json.dumps(line), flush=True)


# The paper's center-outward ranking correlations (Sec. 6): Table 4 (Gaussian, d = 5 ... 150) and Table 5
# (d = 50, Student t with nu = 1, 2, 5, 10), 5,000 points of n = 100,000, k = 100,000 over r = 40, alpha = 0.9.
# Rows: the density against D_P, against D_AP, against the Mahalanobis depth with the sample mean and MLE
# covariance, and D_P against D_AP.  (The robust MCD-based Mahalanobis rows are not reproduced.)
PAPER_RANK_D = (5, 10, 25, 50, 100, 150)
PAPER_RANK_NU = (1, 2, 5, 10)
PAPER_TABLE4 = {
    "spearman": {"pdf_dp": (.9999, .9998, .9995, .9987, .9963, .9912), "pdf_dap": (.9987, .9969, .9903, .9812, .9549, .9140),
                 "pdf_dml": (.9999, .9998, .9998, .9996, .9993, .9990), "dp_dap": (.9987, .9971, .9907, .9810, .9536, .9115)},
    "kendall": {"pdf_dp": (.9929, .9891, .9821, .9687, .9483, .9216), "pdf_dap": (.9697, .9530, .9172, .8820, .8157, .7468),
                "pdf_dml": (.9945, .9921, .9892, .9848, .9793, .9741), "dp_dap": (.9704, .9545, .9187, .8813, .8123, .7431)},
}
PAPER_TABLE5 = {
    "spearman": {"pdf_dp": (.9999, .9998, .9995, .9991), "pdf_dap": (.9996, .9992, .9982, .9967),
                 "pdf_dml": (.9936, .9978, .9999, .9999), "dp_dap": (.9995, .9990, .9978, .9960)},
    "kendall": {"pdf_dp": (.9907, .9871, .9804, .9741), "pdf_dap": (.9836, .9771, .9638, .9514),
                "pdf_dml": (.9332, .9608, .9936, .9934), "dp_dap": (.9817, .9742, .9597, .9461)},
}


def run_ranks(args):
    """Center-outward ordering on the paper's ranking data: D_P and D_AP of points drawn from an n = 100,000
    cloud (keys beyond shared memory, so every selection pass recomputes them), rank-correlated with the
    true density and with the Mahalanobis depth (sample mean, MLE covariance).  The paper's k = 100,000
    directions over r = 40 rounds, alpha = 0.9, on a bounded sample of its 5,000 points: --nq (100);
    --grid-k overrides k."""
    import torch
    from scipy.stats import kendalltau, spearmanr
    from __graft_entry__ import build
    build()
    import paper_2506_08262_gb300 as rrs
    dev = torch.device("cuda", 0)
    ctx = rrs.rrs_create(0, 0)
    stream = torch.cuda.current_stream(dev)
    n, r, alpha = 100_000, 40, 0.9
    npts = args.nq or 100
    k = (args.grid_k or [100_000])[0]
    configs = [(d, np.inf) for d in PAPER_RANK_D if not args.grid_d or d in args.grid_d]
    if not args.grid_d or 50 in args.grid_d:
        configs += [(50, float(nu)) for nu in PAPER_RANK_NU]
    sampler = ClockSampler(0)
    sampler.start()
    rows, total_ms, total_q = [], 0.0, 0
    for ci, (d, nu) in enumerate(configs):
        X, Z, S = workloads.ranking_cloud(600 + ci, n, d, nu, npts)
        did = rrs.rrs_register_dataset(ctx, torch.from_numpy(X).to(dev), n, d, rrs.RRS_F32, True)
        Zd = torch.from_numpy(Z).to(dev)
        depth, ms = {}, {}
        for kind in (workloads.PROJECTION, workloads.ASYM_PROJECTION):
            dep = torch.empty(npts, dtype=torch.float64, device=dev)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            rrs.rrs_depth(ctx, did, Zd, npts, rrs.RRS_F32, True, kind, k, r, alpha, 0, rrs.RRS_PREC_FP32_SIMT,
                          dep, None, None, None, True, stream)
            b.record(stream)
            torch.cuda.synchronize()
            ms[kind] = a.elapsed_time(b)
            depth[kind] = dep.cpu().numpy()
        rrs.rrs_check(ctx, stream)
        rrs.rrs_free(ctx, did)
        # the density is a decreasing function of z' S^-1 z for both families (mean 0, scatter S)
        Zf = Z.astype(np.float64)
        pdf_score = -np.einsum("ij,ij->i", Zf, np.linalg.solve(S, Zf.T).T)
        Xf = X.astype(np.float64)
        mu = Xf.mean(axis=0)
        cov = (Xf - mu).T @ (Xf - mu) / n
        dz = Zf - mu
        dml = 1.0 / (1.0 + np.einsum("ij,ij->i", dz, np.linalg.solve(cov, dz.T).T))
        dp, dap = depth[workloads.PROJECTION], depth[workloads.ASYM_PROJECTION]
        pairs = {"pdf_dp": (pdf_score, dp), "pdf_dap": (pdf_score, dap), "pdf_dml": (pdf_score, dml),
                 "dp_dap": (dp, dap)}
        if np.isfinite(nu):
            paper = {t: {key: PAPER_TABLE5[t][key][PAPER_RANK_NU.index(int(nu))] for key in pairs} for t in PAPER_TABLE5}
        else:
            paper = {t: {key: PAPER_TABLE4[t][key][PAPER_RANK_D.index(d)] for key in pairs} for t in PAPER_TABLE4}
        rows.append({"d": d, "family": "gaussian" if not np.isfinite(nu) else f"student_t_nu{int(nu)}",
                     "spearman": {key: round(float(spearmanr(x, y)[0]), 4) for key, (x, y) in pairs.items()},
                     "kendall": {key: round(float(kendalltau(x, y)[0]), 4) for key, (x, y) in pairs.items()},
                     "paper": paper, "ms": {"projection": round(ms[workloads.PROJECTION], 1),
                                            "asymmetric": round(ms[workloads.ASYM_PROJECTION], 1)}})
        total_ms += ms[workloads.PROJECTION] + ms[workloads.ASYM_PROJECTION]
        total_q += 2 * npts
    clocks = sampler.stop()
    rrs.rrs_destroy(ctx)
    line = {"metric": "center-outward ranking correlation (paper's Sec. 6)", "value": total_q / (total_ms / 1000),
            "unit": "query-depths/s", "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "ranking: n = 100,000 N(0, Toeplitz 2^-|i-j|) (d = 5..150) or multivariate t "
                                   "(nu = 1, 2, 5, 10; d = 50), query points drawn from the cloud, D_P and D_AP "
                                   "with keys recomputed per selection pass",
                       "points": npts, "k": k, "r": r, "alpha": alpha,
                       "paper_run": "5,000 points, k = 100,000 (this run: a bounded sample of points)"},
            "rows": rows, "clocks": clocks}
    print(json.dumps(line), flush=True)


def run_convergence(args):
    """The paper's cap-shrinkage convergence study (Sec. 5.1) for D_P: n = 50,000 normal points in d = 50
    (Toeplitz covariance), --nq points (50) drawn from the cloud, a reference depth per point = the minimum
    over three seeds of r = 100, alpha = 0.9 runs with --grid-k directions (1,000,000; the paper uses
    3,000,000), then the mean squared error to it over alpha in {0.6, 0.7, 0.8, 0.9}, r in {25, 30, 35} and
    k from 200 to 90,000.  All 108 grid cells run as requests of one rrs_depth_batched call."""
    import torch
    from __graft_entry__ import build
    build()
    import paper_2506_08262_gb300 as rrs
    dev = torch.device("cuda", 0)
    ctx = rrs.rrs_create(0, 0)
    stream = torch.cuda.current_stream(dev)
    n, d = 50_000, 50
    npts = args.nq or 50
    k_ref = (args.grid_k or [1_000_000])[0]
    X, Z, _ = workloads.ranking_cloud(700, n, d, np.inf, npts)
    did = rrs.rrs_register_dataset(ctx, torch.from_numpy(X).to(dev), n, d, rrs.RRS_F32, True)
    Zd = torch.from_numpy(Z).to(dev)
    sampler = ClockSampler(0)
    sampler.start()

    def batched(cells):
        outs, reqs = [], []
        for (k, r, alpha, seed) in cells:
            o = torch.empty(npts, dtype=torch.float64, device=dev)
            outs.append(o)
            reqs.append(rrs.rrs_request(dataset_id=did, Z=Zd.data_ptr(), n_queries=npts, dtype=rrs.RRS_F32,
                                        kind=rrs.RRS_PROJECTION, n_dirs=k, n_refinements=r, cap_shrink=alpha,
                                        seed=seed, depth_out=o.data_ptr(), precision=rrs.RRS_PREC_FP32_SIMT))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rrs.rrs_depth_batched(ctx, reqs, use_graph=False, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        rrs.rrs_check(ctx, stream)
        return [o.cpu().numpy() for o in outs], a.elapsed_time(b), sum(k for k, _, _, _ in cells) * npts * n

    ref_runs, ref_ms, ref_pd = batched([(k_ref, 100, 0.9, s) for s in (101, 102, 103)])
    ref = np.minimum.reduce(ref_runs)
    alphas, rs, ks = (0.6, 0.7, 0.8, 0.9), (25, 30, 35), (200, 500, 1_000, 2_000, 5_000, 10_000, 20_000, 50_000, 90_000)
    cells = [(k, r, a, 7) for a in alphas for r in rs for k in ks]
    got, grid_ms, grid_pd = batched(cells)
    clocks = sampler.stop()
    rrs.rrs_free(ctx, did)
    rrs.rrs_destroy(ctx)
    mse = {}
    below = 0
    for (k, r, a, _), g in zip(cells, got):
        mse.setdefault(f"alpha={a}", {}).setdefault(f"r={r}", {})[k] = float(np.mean((g - ref) ** 2))
        below += int(np.sum(g < ref))
    # the paper's reading of its figure: larger alpha converges faster; summarised here per alpha as the
    # mean over r of the MSE at each k
    by_alpha = {a: [float(np.mean([mse[a][rk][k] for rk in mse[a]])) for k in ks] for a in mse}
    line = {"metric": "convergence of D_P to the reference depth (paper's Sec. 5.1)", "value": float(by_alpha["alpha=0.9"][-1]),
            "unit": "mean squared error at alpha = 0.9, k = 90,000 (mean over r)", "n_gpus": 1,
            "higher_is_better": False, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "convergence: n = 50,000 N(0, Toeplitz 2^-|i-j|), d = 50, points drawn from "
                                   "the cloud, D_P; grid alpha x r x k in one batched call",
                       "points": npts, "reference": {"k": k_ref, "r": 100, "alpha": 0.9, "seeds": 3,
                                                     "paper": "k = 3,000,000"},
                       "grid": {"alpha": alphas, "r": rs, "k": ks}},
            "mse_by_alpha_mean_over_r": {"k": ks, **by_alpha}, "mse": mse,
            "grid_depths_below_reference": below,
            "timing": {"reference_s": ref_ms / 1000, "reference_pd_per_s": ref_pd / (ref_ms / 1000),
                       "grid_s": grid_ms / 1000, "grid_pd_per_s": grid_pd / (grid_ms / 1000)},
            "clocks": clocks}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "c1":
        run_c1(args)
    elif args.workload == "c3":
        run_c3(args)
    elif args.workload == "c4":
        run_c4(args)
    elif args.workload == "c5":
        run_c5(args)
    elif args.workload == "grid":
        run_grid(args)
    elif args.workload == "ranks":
        run_ranks(args)
    elif args.workload == "convergence":
        run_convergence(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
