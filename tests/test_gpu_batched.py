"""Batched multi-dataset launches (rrs_depth_batched) on the GPU.

Many independent requests -- datasets of uneven n and d, each with its own
queries, depth kind and round count -- share every launch of a round.  Each
query keeps its own direction stream and its own dataset's statistics, so a
request's results must equal those of rrs_depth on that request alone, bit for
bit, with or without the captured-graph replay; a sample is also checked against
the CPU oracle.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2506_08262_gb300 as rrs
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from __graft_entry__ import build
    build()
    c = rrs.Context(0)
    yield c
    c.close()


def make_requests(ctx, problems, r_override=None):
    reqs, outs, ids = [], [], []
    for i, P in enumerate(problems):
        did = ctx.register(torch.from_numpy(P.X).cuda())
        ids.append(did)
        Z = torch.from_numpy(P.Z).cuda()
        r = P.r if r_override is None else r_override[i]
        o = {"Z": Z, "depth": torch.full((P.nq,), -1.0, dtype=torch.float64, device="cuda"),
             "count": torch.zeros(P.nq, dtype=torch.int64, device="cuda"),
             "best": torch.zeros(P.nq, dtype=torch.int32, device="cuda"),
             "choice": torch.zeros((P.nq, r), dtype=torch.int32, device="cuda"), "r": r}
        req = rrs.rrs_request(dataset_id=did, Z=Z.data_ptr(), n_queries=P.nq, dtype=rrs.RRS_F32, kind=P.kind,
                              n_dirs=P.k, n_refinements=r, cap_shrink=P.alpha, seed=P.seed + i,
                              depth_out=o["depth"].data_ptr(), count_out=o["count"].data_ptr(),
                              best_out=o["best"].data_ptr(), round_choice_out=o["choice"].data_ptr())
        reqs.append(req)
        outs.append(o)
    return reqs, outs, ids


def alone(ctx, did, P, r, seed, Z):
    dep, cnt, best, ch = ctx.depth(did, Z, P.kind, P.k, r, P.alpha, seed, rounds=True)
    return dep.cpu().numpy(), cnt.cpu().numpy(), best.cpu().numpy(), ch.cpu().numpy()


@pytest.mark.parametrize("use_graph", [False, True])
def test_batched_equals_alone(ctx, use_graph):
    problems = workloads.c4(seed=41, n_datasets=12, n_lo=50, n_hi=3000, q_hi=20, scale=1.0)
    for P in problems:
        P.k, P.r = 120, 4
    # uneven round counts: requests leave the batch at different rounds
    r_override = [4, 2, 3, 4, 1, 4, 2, 3, 4, 4, 1, 2]
    reqs, outs, ids = make_requests(ctx, problems, r_override)
    stream = torch.cuda.current_stream()
    for rep in range(2 if use_graph else 1):
        rrs.rrs_depth_batched(ctx.handle, reqs, use_graph=use_graph, stream=stream)
        rrs.rrs_check(ctx.handle, stream)
        for i, P in enumerate(problems):
            d, c, b, ch = alone(ctx, ids[i], P, outs[i]["r"], P.seed + i, outs[i]["Z"])
            np.testing.assert_array_equal(outs[i]["depth"].cpu().numpy(), d)
            np.testing.assert_array_equal(outs[i]["best"].cpu().numpy(), b)
            np.testing.assert_array_equal(outs[i]["choice"].cpu().numpy(), ch)
            if P.kind == 0:
                np.testing.assert_array_equal(outs[i]["count"].cpu().numpy(), c)
    for did in ids:
        ctx.free(did)


def test_batched_mixes_outside_and_resident_keys(ctx):
    # datasets whose keys exceed shared memory (kept in device memory) batched with resident-key ones:
    # each request's results equal its rrs_depth call alone
    problems = []
    for i, (n, d, kind) in enumerate([(60_000, 6, 1), (2_000, 6, 1), (61_003, 20, 2), (900, 20, 2), (3_000, 5, 0)]):
        X, Z = workloads.gaussian_cloud(200 + i, n, d, 3, dtype=np.float32)
        problems.append(workloads.Problem(X, Z, kind, 60, 3, 0.8, 0))
    reqs, outs, ids = make_requests(ctx, problems)
    stream = torch.cuda.current_stream()
    rrs.rrs_depth_batched(ctx.handle, reqs, use_graph=False, stream=stream)
    rrs.rrs_check(ctx.handle, stream)
    for i, P in enumerate(problems):
        d, c, b, ch = alone(ctx, ids[i], P, P.r, P.seed + i, outs[i]["Z"])
        np.testing.assert_array_equal(outs[i]["depth"].cpu().numpy(), d)
        np.testing.assert_array_equal(outs[i]["best"].cpu().numpy(), b)
        np.testing.assert_array_equal(outs[i]["choice"].cpu().numpy(), ch)
    for did in ids:
        ctx.free(did)


def test_batched_mixes_staged_and_in_place_directions(ctx):
    # one launch generates d = 10 directions in shared memory and d = 200 ones in place in device memory
    problems = []
    for i, (n, d, kind) in enumerate([(400, 200, 0), (900, 10, 1), (500, 200, 2), (700, 10, 0)]):
        X, Z = workloads.gaussian_cloud(250 + i, n, d, 4, dtype=np.float32)
        problems.append(workloads.Problem(X, Z, kind, 60, 3, 0.8, 0))
    reqs, outs, ids = make_requests(ctx, problems)
    stream = torch.cuda.current_stream()
    rrs.rrs_depth_batched(ctx.handle, reqs, use_graph=False, stream=stream)
    rrs.rrs_check(ctx.handle, stream)
    for i, P in enumerate(problems):
        d, c, b, ch = alone(ctx, ids[i], P, P.r, P.seed + i, outs[i]["Z"])
        np.testing.assert_array_equal(outs[i]["depth"].cpu().numpy(), d)
        np.testing.assert_array_equal(outs[i]["best"].cpu().numpy(), b)
        np.testing.assert_array_equal(outs[i]["choice"].cpu().numpy(), ch)
        if P.kind == 0:
            np.testing.assert_array_equal(outs[i]["count"].cpu().numpy(), c)
    for did in ids:
        ctx.free(did)


def test_batched_against_oracle_sample(ctx):
    problems = workloads.c4(seed=43, n_datasets=6, n_lo=100, n_hi=2000, q_hi=6, scale=1.0)
    for P in problems:
        P.k, P.r = 60, 3
    reqs, outs, ids = make_requests(ctx, problems)
    rrs.rrs_depth_batched(ctx.handle, reqs, stream=torch.cuda.current_stream())
    rrs.rrs_check(ctx.handle, torch.cuda.current_stream())
    for i, P in enumerate(problems):
        got = outs[i]["depth"].cpu().numpy()
        if P.kind == 0:
            ref = oracle.rrs(P.X, P.Z, 0, P.k, P.r, P.alpha, P.seed + i)
            np.testing.assert_array_equal(outs[i]["count"].cpu().numpy(), ref["count"])
        else:
            ref = oracle.rrs(P.X, P.Z, P.kind, P.k, P.r, P.alpha, P.seed + i,
                             follow=outs[i]["choice"].cpu().numpy())
            np.testing.assert_allclose(got, ref["depth"], rtol=1e-5)
    for did in ids:
        ctx.free(did)


def test_batched_rejects_bad_request(ctx):
    X = torch.zeros((5, 3), dtype=torch.float32, device="cuda")
    did = ctx.register(X)
    Z = torch.zeros((2, 3), dtype=torch.float32, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    bad = rrs.rrs_request(dataset_id=did, Z=Z.data_ptr(), n_queries=2, dtype=rrs.RRS_F32, kind=1, n_dirs=3,
                          n_refinements=5, cap_shrink=0.5, seed=0, depth_out=out.data_ptr())
    with pytest.raises(rrs.RRSError) as e:
        rrs.rrs_depth_batched(ctx.handle, [bad])
    assert e.value.status == rrs.RRS_ERR_INVALID_ARG
    ctx.free(did)


def test_batched_tensor_core_halfspace(ctx):
    # halfspace requests on the tensor cores inside a mixed batch (datasets of uneven n and d,
    # d on both sides of the 64-wide K extent): results equal rrs_depth alone at the same
    # precision, and the counts equal the FP32 path's
    problems = workloads.c4(seed=47, n_datasets=8, n_lo=100, n_hi=3000, q_hi=12, scale=1.0)
    for i, P in enumerate(problems):
        P.k, P.r = 150, 3
        P.kind = 0 if i % 3 != 2 else 1
    reqs, outs, ids = make_requests(ctx, problems)
    for i, P in enumerate(problems):
        if P.kind == 0:
            reqs[i].precision = rrs.RRS_PREC_SPLIT_BF16X3
    for use_graph in (False, True):
        rrs.rrs_depth_batched(ctx.handle, reqs, use_graph=use_graph, stream=torch.cuda.current_stream())
        rrs.rrs_check(ctx.handle, torch.cuda.current_stream())
        for i, P in enumerate(problems):
            prec = reqs[i].precision
            dep, cnt, best, ch = ctx.depth(ids[i], outs[i]["Z"], P.kind, P.k, P.r, P.alpha, P.seed + i,
                                           precision=prec, rounds=True)
            np.testing.assert_array_equal(outs[i]["depth"].cpu().numpy(), dep.cpu().numpy())
            np.testing.assert_array_equal(outs[i]["choice"].cpu().numpy(), ch.cpu().numpy())
            if P.kind == 0:
                np.testing.assert_array_equal(outs[i]["count"].cpu().numpy(), cnt.cpu().numpy())
                d32, c32, _, _ = ctx.depth(ids[i], outs[i]["Z"], 0, P.k, P.r, P.alpha, P.seed + i, rounds=True)
                np.testing.assert_array_equal(outs[i]["count"].cpu().numpy(), c32.cpu().numpy())
    # one tensor-core launch per round and K extent of the planes (64 or 128), whatever the datasets: each
    # CTA takes its dataset's tensor map from the device table
    kps = {64 if P.d + 2 <= 64 else 128 for P in problems if P.kind == 0}
    rrs.rrs_profile_enable(ctx.handle, True)
    rrs.rrs_depth_batched(ctx.handle, reqs, use_graph=False, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    prof = rrs.rrs_profile_read(ctx.handle)
    rrs.rrs_profile_enable(ctx.handle, False)
    rounds = max(P.r for P in problems if P.kind == 0)
    assert prof["hd_tc"][1] == rounds * len(kps), (prof["hd_tc"], kps)
    for did in ids:
        ctx.free(did)


def test_batched_rejects_tensor_cores_for_projection_depth(ctx):
    X = torch.zeros((5, 3), dtype=torch.float32, device="cuda")
    did = ctx.register(X)
    Z = torch.zeros((2, 3), dtype=torch.float32, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    bad = rrs.rrs_request(dataset_id=did, Z=Z.data_ptr(), n_queries=2, dtype=rrs.RRS_F32, kind=1, n_dirs=4,
                          n_refinements=2, cap_shrink=0.5, seed=0, depth_out=out.data_ptr(),
                          precision=rrs.RRS_PREC_SPLIT_BF16X3)
    with pytest.raises(rrs.RRSError) as e:
        rrs.rrs_depth_batched(ctx.handle, [bad])
    assert e.value.status == rrs.RRS_ERR_INVALID_ARG
    ctx.free(did)
