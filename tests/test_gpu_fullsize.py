"""Full-size parity: the projection-depth and halfspace workloads at the sizes the
benchmark times (same dataset sizes, directions and rounds, same entry point and
kernel choice), every query computed on the GPU, a sample of queries recomputed
by the CPU oracle with the same direction-stream counters.

Halfspace counts must match bit for bit; projection and asymmetric projection
depths in follow mode within 1e-5 relative (see test_gpu_parity.py).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2506_08262_gb300 as rrs
import workloads
from test_gpu_parity import H, P, AP, assert_follow, assert_hd_exact, gpu_rrs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from __graft_entry__ import build
    build()
    c = rrs.Context(0)
    yield c
    c.close()


def sub(g, idx):
    return {k: v[idx] for k, v in g.items()}


@pytest.mark.parametrize("kind", [P, AP])
def test_projection_workload_full_size_sampled(ctx, kind):
    # n = 10,000, d = 10, 1,000 queries, k = 1,000 over r = 20, tuned group size as in the benchmark
    Pr = workloads.c2(kind=kind)
    did = ctx.register(torch.from_numpy(Pr.X).cuda())
    try:
        rrs.rrs_autotune(ctx.handle, did, kind, Pr.k, Pr.r)
        dep, cnt, best, ch = ctx.depth(did, torch.from_numpy(Pr.Z).cuda(), kind, Pr.k, Pr.r, Pr.alpha, Pr.seed,
                                       rounds=True)
        g = {"depth": dep.cpu().numpy(), "count": cnt.cpu().numpy(), "best": best.cpu().numpy(),
             "choice": ch.cpu().numpy()}
    finally:
        ctx.free(did)
    assert np.all((g["depth"] >= 0) & (g["depth"] <= 1))
    idx = np.array([0, 137, 500, 999])
    assert_follow(sub(g, idx), Pr.X, Pr.Z[idx], kind, Pr.k, Pr.r, Pr.alpha, Pr.seed, qidx=idx)


def test_halfspace_workload_full_size_sampled(ctx):
    # n = 100,000 Student-t rows in d = 50, k = 2,000 over r = 20; two launch waves of queries on the
    # tensor cores, the FP32 path on the same queries, three queries recomputed exactly by the oracle
    Pr = workloads.c3(nq=304)
    tc = gpu_rrs(ctx, Pr.X, Pr.Z, H, Pr.k, Pr.r, Pr.alpha, Pr.seed, precision=rrs.RRS_PREC_SPLIT_BF16X3)
    f32 = gpu_rrs(ctx, Pr.X, Pr.Z, H, Pr.k, Pr.r, Pr.alpha, Pr.seed)
    for key in ("count", "depth", "best", "choice"):
        np.testing.assert_array_equal(tc[key], f32[key])
    idx = np.array([0, 151, 303])
    ref = oracle.rrs(Pr.X, Pr.Z[idx], H, Pr.k, Pr.r, Pr.alpha, Pr.seed, qidx=idx)
    assert_hd_exact(sub(tc, idx), ref)
