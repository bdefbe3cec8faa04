"""Serving loop (continuous batching) on the GPU.

Requests are admitted into a fixed pool of query slots as slots free up and
each step runs one refinement round for every active query, so requests that
arrive while others are in flight share the same launches.  A request's depths
must not depend on the mix: they must equal rrs_depth on that request alone,
bit for bit, whether it was served alone, between others, or after waiting for
slots; one halfspace request is also checked against the CPU oracle.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2506_08262_gb300 as rrs
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from __graft_entry__ import build
    build()
    ctx = rrs.Context(0)
    datasets = []
    for i, P in enumerate(workloads.c4(seed=51, n_datasets=5, n_lo=200, n_hi=4000, q_hi=40)):
        did = ctx.register(torch.from_numpy(P.X).cuda())
        datasets.append((did, P))
    yield ctx, datasets
    for did, _ in datasets:
        ctx.free(did)
    ctx.close()


K, R, ALPHA = 120, 4, 0.8


def serve(ctx, batches, max_slots=4096, precision=rrs.RRS_PREC_FP32_SIMT, work_limit=None, steps_out=None):
    """batches: list (one per step) of lists of (dataset_id, Z, kind, seed) to submit before that step."""
    srv = rrs.rrs_server_create(ctx.handle, max_slots, -(-K // R), 100, torch.cuda.current_stream(),
                                precision=precision)
    if work_limit is not None:
        rrs.rrs_server_set_work_limit(srv, work_limit)
    results, pending = [], {}
    try:
        step = 0
        while step < len(batches) or pending:
            if step < len(batches):
                for did, Z, kind, seed in batches[step]:
                    out = np.full(Z.shape[0], -1.0)
                    rid = rrs.rrs_server_submit(srv, did, Z, Z.shape[0], rrs.RRS_F32, kind, K, R, ALPHA, seed, out)
                    pending[rid] = out
                    results.append(out)
            rrs.rrs_server_step(srv)
            for rid in list(pending):
                if rrs.rrs_server_poll(srv, rid):
                    del pending[rid]
            step += 1
            assert step < 10_000
        torch.cuda.synchronize()
        rrs.rrs_check(ctx.handle, torch.cuda.current_stream())
        if steps_out is not None:
            steps_out.append(step)
    finally:
        rrs.rrs_server_destroy(srv)
    return results


def alone_depth(ctx, did, Z, kind, seed, precision=rrs.RRS_PREC_FP32_SIMT):
    prec = precision if kind == 0 else rrs.RRS_PREC_FP32_SIMT
    dep, _, _ = ctx.depth(did, torch.from_numpy(Z).cuda(), kind, K, R, ALPHA, seed, precision=prec)
    return dep.cpu().numpy()


def test_same_result_alone_and_in_the_mix(setup):
    ctx, ds = setup
    rng = np.random.default_rng(0)
    target = (ds[2][0], np.ascontiguousarray(ds[2][1].Z[:7]), 1, 99)
    others = []
    for i in range(12):
        did, P = ds[i % len(ds)]
        q = int(rng.integers(1, P.nq + 1))
        others.append((did, np.ascontiguousarray(P.Z[:q]), i % 3, 1000 + i))
    a = serve(ctx, [[target]])[0]
    # the target arrives at step 2, while earlier requests are mid-flight, and more follow
    mix = serve(ctx, [others[:4], others[4:6], [target] + others[6:9], others[9:]])
    b = mix[6]
    ref = alone_depth(ctx, target[0], target[1], target[2], target[3])
    np.testing.assert_array_equal(a, ref)
    np.testing.assert_array_equal(b, ref)
    # every request of the mix equals its alone result
    flat = others[:4] + others[4:6] + [target] + others[6:9] + others[9:]
    for (did, Z, kind, seed), got in zip(flat, mix):
        np.testing.assert_array_equal(got, alone_depth(ctx, did, Z, kind, seed))


def test_requests_wait_for_slots(setup):
    ctx, ds = setup
    reqs = []
    for i in range(10):
        did, P = ds[i % len(ds)]
        reqs.append((did, np.ascontiguousarray(P.Z[: min(P.nq, 20)]), i % 3, 7 + i))
    got = serve(ctx, [reqs], max_slots=40)   # far fewer slots than queries: requests queue
    for (did, Z, kind, seed), g in zip(reqs, got):
        np.testing.assert_array_equal(g, alone_depth(ctx, did, Z, kind, seed))


def test_served_halfspace_matches_oracle(setup):
    ctx, ds = setup
    did, P = ds[0]
    Z = np.ascontiguousarray(P.Z[:5])
    got = serve(ctx, [[(did, Z, 0, 5)]])[0]
    ref = oracle.rrs(P.X, Z, 0, K, R, ALPHA, 5)
    np.testing.assert_array_equal(got, ref["depth"])


def test_oversize_request_is_rejected(setup):
    ctx, ds = setup
    did, P = ds[0]
    srv = rrs.rrs_server_create(ctx.handle, 4, 30, 100, torch.cuda.current_stream())
    try:
        Z = np.ascontiguousarray(P.Z[:5])
        with pytest.raises(rrs.RRSError) as e:
            rrs.rrs_server_submit(srv, did, Z, 5, rrs.RRS_F32, 0, K, R, ALPHA, 0, np.zeros(5))
        assert e.value.status == rrs.RRS_ERR_UNSUPPORTED
    finally:
        rrs.rrs_server_destroy(srv)


def test_tensor_core_server_same_alone_and_in_the_mix(setup):
    # halfspace requests served on the tensor cores: each result equals rrs_depth alone at the
    # same precision, and (counts being exact) the FP32 server's result
    ctx, ds = setup
    TCP = rrs.RRS_PREC_SPLIT_BF16X3
    rng = np.random.default_rng(3)
    reqs = []
    for i in range(9):
        did, P = ds[i % len(ds)]
        q = int(rng.integers(1, min(P.nq, 25) + 1))
        reqs.append((did, np.ascontiguousarray(P.Z[:q]), 0 if i % 3 else 1 + (i % 2), 300 + i))
    mix = serve(ctx, [reqs[:3], reqs[3:5], reqs[5:]], precision=TCP)
    fp32 = serve(ctx, [reqs[:3], reqs[3:5], reqs[5:]])
    for (did, Z, kind, seed), got, ref32 in zip(reqs, mix, fp32):
        np.testing.assert_array_equal(got, alone_depth(ctx, did, Z, kind, seed, precision=TCP))
        np.testing.assert_array_equal(got, ref32)


def test_served_keys_beyond_shared_memory(setup):
    # a projection-depth request on a dataset too large for resident keys, served between small ones
    ctx, ds = setup
    X, Zb = workloads.gaussian_cloud(57, 57_000, 8, 4, dtype=np.float32)
    big = ctx.register(torch.from_numpy(X).cuda())
    try:
        reqs = [(ds[0][0], np.ascontiguousarray(ds[0][1].Z[:3]), 1, 11), (big, np.ascontiguousarray(Zb), 1, 12),
                (big, np.ascontiguousarray(Zb[:2]), 2, 13), (ds[1][0], np.ascontiguousarray(ds[1][1].Z[:3]), 2, 14)]
        got = serve(ctx, [reqs[:2], reqs[2:]])
        for (did, Z, kind, seed), g in zip(reqs, got):
            np.testing.assert_array_equal(g, alone_depth(ctx, did, Z, kind, seed))
    finally:
        ctx.free(big)


@pytest.mark.parametrize("work_limit", [1.0, 2e5, 0.0])
def test_work_limit_changes_the_steps_not_the_results(setup, work_limit):
    # the work limit bounds the queries that run a round in one step (at least one query); 0 runs every
    # admitted query at every step.  A limit of one pair runs one query per step, so every query's R rounds
    # take a step of their own.  Results equal rrs_depth alone whatever the limit.
    ctx, ds = setup
    batch = []
    for i in range(4):
        did, P = ds[i]
        batch.append((did, np.ascontiguousarray(P.Z[:3 + i]), i % 3, 300 + i))
    steps = []
    res = serve(ctx, [batch], work_limit=work_limit, steps_out=steps)
    for (did, Z, kind, seed), got in zip(batch, res):
        np.testing.assert_array_equal(got, alone_depth(ctx, did, Z, kind, seed))
    total_q = sum(Z.shape[0] for _, Z, _, _ in batch)
    if work_limit == 1.0:
        assert steps[0] >= total_q * R
    if work_limit == 0.0:
        assert steps[0] <= R + 1


def test_work_limit_rejects_bad_values(setup):
    ctx, _ = setup
    srv = rrs.rrs_server_create(ctx.handle, 16, 30, 100, torch.cuda.current_stream())
    try:
        for bad in (-1.0, float("nan"), float("inf")):
            with pytest.raises(rrs.RRSError) as e:
                rrs.rrs_server_set_work_limit(srv, bad)
            assert e.value.status == rrs.RRS_ERR_INVALID_ARG
    finally:
        rrs.rrs_server_destroy(srv)
