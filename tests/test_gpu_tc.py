"""GPU parity of the tensor-core halfspace path (tcgen05, split-BF16x3 products).

Halfspace counts are exact whatever the projection arithmetic, because every
point in the near-tie band is re-checked with an exact sign test; so the
tensor-core path must reproduce the CPU oracle bit for bit, and the FP32 path
as well.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2506_08262_gb300 as rrs
import workloads

pytestmark = pytest.mark.gpu

H = 0
TC = rrs.RRS_PREC_SPLIT_BF16X3


@pytest.fixture(scope="module")
def ctx():
    from __graft_entry__ import build
    build()
    c = rrs.Context(0)
    yield c
    c.close()


def run(ctx, X, Z, k, r, alpha, seed, precision):
    did = ctx.register(torch.from_numpy(X).cuda())
    try:
        dep, cnt, best, ch = ctx.depth(did, torch.from_numpy(Z).cuda(), H, k, r, alpha, seed, precision=precision,
                                       rounds=True)
        return {"depth": dep.cpu().numpy(), "count": cnt.cpu().numpy(), "best": best.cpu().numpy(),
                "choice": ch.cpu().numpy()}
    finally:
        ctx.free(did)


def test_tc_tiny_case_matches_oracle(ctx):
    X, Z = workloads.gaussian_cloud(77, 300, 5, 2, dtype=np.float32)
    g = run(ctx, X, Z, 20, 2, 0.5, 3, TC)
    ref = oracle.rrs(X, Z, H, 20, 2, 0.5, 3)
    np.testing.assert_array_equal(g["count"], ref["count"])
    np.testing.assert_array_equal(g["best"], ref["best"])


@pytest.mark.parametrize("n,d,dtype", [(1, 1, np.float32), (129, 2, np.float64), (1000, 10, np.float32),
                                       (3001, 50, np.float32), (2500, 62, np.float32), (1537, 100, np.float32),
                                       (777, 126, np.float64)])
def test_tc_halfspace_bit_exact(ctx, n, d, dtype):
    X, Z = workloads.gaussian_cloud(n * 7 + d, n, d, 5, dtype=dtype, zscale=1.3)
    Z[0] = X[0]
    g = run(ctx, X, Z, 300, 3, 0.7, 11, TC)
    ref = oracle.rrs(X, Z, H, 300, 3, 0.7, 11)
    np.testing.assert_array_equal(g["count"], ref["count"])
    np.testing.assert_array_equal(g["depth"], ref["depth"])
    np.testing.assert_array_equal(g["best"], ref["best"])


def test_tc_equals_fp32_path_on_heavy_tails(ctx):
    P = workloads.c3(n=4000, nq=12)
    a = run(ctx, P.X, P.Z, 400, 4, P.alpha, 0, TC)
    b = run(ctx, P.X, P.Z, 400, 4, P.alpha, 0, rrs.RRS_PREC_FP32_SIMT)
    for key in ("count", "depth", "best", "choice"):
        np.testing.assert_array_equal(a[key], b[key])


def test_tc_round_counts_exact_and_band_sound(ctx):
    # per-direction counts for caller-supplied directions against the oracle, plus the
    # number of near-tie re-checks (every point whose fast sign could be wrong is in the band)
    P = workloads.c3(n=2049, nq=3)
    m = 128
    U = np.stack([oracle.directions(5, q, 0, m, P.d, 0.9) for q in range(3)])
    did = ctx.register(torch.from_numpy(P.X).cuda())
    dep = torch.empty((3, m), dtype=torch.float64, device="cuda")
    cnt = torch.empty((3, m), dtype=torch.int64, device="cuda")
    band = torch.zeros(3, dtype=torch.int64, device="cuda")
    rrs.rrs_debug_round_depths(ctx.handle, did, torch.from_numpy(P.Z).cuda(), 3, rrs.RRS_F32, H, m,
                               torch.from_numpy(U).cuda(), TC, dep, cnt, band)
    ctx.free(did)
    c = cnt.cpu().numpy()
    for q in range(3):
        for j in range(0, m, 7):
            assert c[q, j] == oracle.univariate(H, P.X, P.Z[q], U[q, j])[1]
    # band re-checks are a small fraction of all point-direction pairs
    assert int(band.sum()) < 0.02 * 3 * m * P.n


@pytest.mark.parametrize("k,r,nq", [(111, 3, 9), (600, 2, 3), (256, 2, 7)])
def test_tc_rows_span_queries(ctx, k, r, nq):
    # a CTA's 128 accumulator rows are consecutive (query, direction) pairs: m = 37 packs
    # several queries per tile, m = 300 starts tiles inside a query, m = 128 fills tiles exactly
    X, Z = workloads.gaussian_cloud(900 + k, 1000, 50, nq, dtype=np.float32, zscale=1.2)
    g = run(ctx, X, Z, k, r, 0.8, 21, TC)
    ref = oracle.rrs(X, Z, H, k, r, 0.8, 21)
    np.testing.assert_array_equal(g["count"], ref["count"])
    np.testing.assert_array_equal(g["best"], ref["best"])
    f = run(ctx, X, Z, k, r, 0.8, 21, rrs.RRS_PREC_FP32_SIMT)
    np.testing.assert_array_equal(g["choice"], f["choice"])


def test_tc_exact_ties_on_a_lattice(ctx):
    # duplicated lattice points and queries placed on data points: many projection
    # differences are exactly zero, so the exact fallback decides them
    rng = np.random.default_rng(8)
    base = rng.integers(-3, 4, size=(150, 6)).astype(np.float32)
    X = np.concatenate([base, base[:90], base[:40]]).astype(np.float32)
    Z = np.concatenate([X[[0, 5, 17, 151]], rng.integers(-3, 4, size=(3, 6)).astype(np.float32)])
    g = run(ctx, X, Z, 200, 2, 0.6, 4, TC)
    ref = oracle.rrs(X, Z, H, 200, 2, 0.6, 4)
    np.testing.assert_array_equal(g["count"], ref["count"])
    np.testing.assert_array_equal(g["depth"], ref["depth"])


def test_tensor_core_tile_width_does_not_change_counts(ctx):
    # planes of K extent 64 run with 256- or 128-point tiles (fixed, tuned or default); counts are exact either
    # way, so every width gives the FP32 path's counts, and a graph captured at one width is dropped when the
    # width changes
    X, Z = workloads.gaussian_cloud(77, 3001, 30, 9, dtype=np.float32)
    did = ctx.register(torch.from_numpy(X).cuda())
    Zt = torch.from_numpy(Z).cuda()
    _, c32, _ = ctx.depth(did, Zt, rrs.RRS_HALFSPACE, 300, 3, 0.6, 5)
    got = {}
    for width in (0, 128, 256, 0):
        rrs.rrs_select_tc_tile(ctx.handle, did, width)
        _, c, _ = ctx.depth(did, Zt, rrs.RRS_HALFSPACE, 300, 3, 0.6, 5, precision=rrs.RRS_PREC_SPLIT_BF16X3)
        got[width] = c.cpu().numpy()
        np.testing.assert_array_equal(got[width], c32.cpu().numpy())
    choice = rrs.rrs_autotune(ctx.handle, did, rrs.RRS_HALFSPACE, 300, 3)
    assert choice in (128, 256)
    # batched with graph replay, before and after a width change
    out = torch.zeros(Z.shape[0], dtype=torch.int64, device="cuda")
    dep = torch.zeros(Z.shape[0], dtype=torch.float64, device="cuda")
    req = rrs.rrs_request(dataset_id=did, Z=Zt.data_ptr(), n_queries=Z.shape[0], dtype=rrs.RRS_F32,
                          kind=rrs.RRS_HALFSPACE, n_dirs=300, n_refinements=3, cap_shrink=0.6, seed=5,
                          depth_out=dep.data_ptr(), count_out=out.data_ptr(), precision=rrs.RRS_PREC_SPLIT_BF16X3)
    for width in (128, 256):
        rrs.rrs_select_tc_tile(ctx.handle, did, width)
        for _ in range(2):
            out.zero_()
            rrs.rrs_depth_batched(ctx.handle, [req], use_graph=True, stream=torch.cuda.current_stream())
            rrs.rrs_check(ctx.handle, torch.cuda.current_stream())
            np.testing.assert_array_equal(out.cpu().numpy(), c32.cpu().numpy())
    rrs.rrs_select_tc_tile(ctx.handle, did, 0)
    ctx.free(did)


def test_tensor_core_tile_choices_by_dimension(ctx):
    # only planes of K extent 64 (d + 2 <= 64) have two tile widths; d + 2 in (64, 128] has 128; larger d has no
    # tensor-core path
    for d, want in ((100, {128}), (140, {0})):
        X, _ = workloads.gaussian_cloud(d, 500, d, 1, dtype=np.float32)
        did = ctx.register(torch.from_numpy(X).cuda())
        assert rrs.rrs_autotune(ctx.handle, did, rrs.RRS_HALFSPACE, 100, 2) in want
        ctx.free(did)
