"""Multi-rank logic of bench.py on CPU (gloo, world size 2).

The path shards by query with no data exchange: every rank holds the data
cloud and takes its own queries, so the benchmark's only cross-rank step is
taking the slowest rank's time and summing the ranks' work.  These tests run
that logic on two gloo ranks.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r'''
import os, sys, json
sys.path.insert(0, os.environ["ROOT"])
import torch.distributed as dist
dist.init_process_group("gloo")
import bench
rank = dist.get_rank()
ms = 10.0 + 5.0 * rank
agg = bench.aggregate_over_ranks(ms)
val = bench.job_value(2000, dist.get_world_size(), agg)
print(json.dumps({"rank": rank, "agg": agg, "value": val}), flush=True)
dist.barrier()
dist.destroy_process_group()
'''


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_take_the_slowest_time():
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, ROOT=ROOT, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=180)
        assert p.returncode == 0, err
        outs.append(out.strip().splitlines()[-1])
    import json
    res = [json.loads(o) for o in outs]
    for r in res:
        assert r["agg"] == 15.0                     # max over ranks
        assert r["value"] == pytest.approx(2 * 2000 / 0.015)


def test_reference_arm_only_rank0_runs(tmp_path):
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_reference_arm_line_carries_the_contract_keys():
    # the oracle arm on the host cores: one JSON line with the metric, a cpu_baseline describing the run and
    # an e2e object without host-device copies
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    assert line["value"] > 0 and line["unit"] == "query-depths/s" and line["higher_is_better"] is True
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"].startswith("projection + asymmetric projection depth")


SHARD_WORKER = r'''
import os, sys, json
sys.path.insert(0, os.environ["ROOT"])
import numpy as np
import torch.distributed as dist
dist.init_process_group("gloo")
import workloads
rank = dist.get_rank()
Z = workloads.c2_queries(rank, 300)
shards = [None, None]
dist.all_gather_object(shards, Z.tolist())
print(json.dumps({"rank": rank, "ok": True}), flush=True)
if rank == 0:
    a, b = np.array(shards[0], np.float32), np.array(shards[1], np.float32)
    assert a.shape == b.shape == (300, 10)
    assert np.array_equal(a, workloads.c2(nq=300).Z)              # rank 0: the workload's own queries
    assert not (a[:, None, :] == b[None, :, :]).all(axis=2).any()  # no query repeats across ranks
    assert b.min() >= -4.0 and b.max() <= 4.0 and abs(float(b.mean())) < 0.3   # same law U[-4,4]^10
dist.barrier()
dist.destroy_process_group()
'''


def test_two_gloo_ranks_take_disjoint_query_shards():
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, ROOT=ROOT, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", SHARD_WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    for p in procs:
        out, err = p.communicate(timeout=180)
        assert p.returncode == 0, err
