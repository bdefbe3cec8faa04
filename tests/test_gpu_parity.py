"""GPU parity: the sm_103a library through its C ABI against the CPU oracle.

Halfspace results must match bit for bit (counts, depths, best directions and
per-round pole choices: counts are exact on both sides, so the whole search
trajectory coincides).  Projection and asymmetric projection depths are
computed from FP32 projections on the GPU and FP64 ones in the oracle; they
are compared in follow mode: the oracle replays the GPU's pole choices and
every round choice and the final depth must agree within 1e-5 relative.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2506_08262_gb300 as rrs
import workloads

pytestmark = pytest.mark.gpu

H, P, AP = 0, 1, 2
TOL = 1e-5


@pytest.fixture(scope="module")
def ctx():
    from __graft_entry__ import build
    build()
    c = rrs.Context(0)
    yield c
    c.close()


def gpu_rrs(ctx, X, Z, kind, k, r, alpha, seed=0, precision=rrs.RRS_PREC_FP32_SIMT, on_device=True):
    did = ctx.register(torch.from_numpy(X).cuda() if on_device else torch.from_numpy(X))
    try:
        Zt = torch.from_numpy(Z).cuda() if on_device else torch.from_numpy(Z)
        dep, cnt, best, ch = ctx.depth(did, Zt, kind, k, r, alpha, seed, precision=precision, rounds=True)
        return {"depth": dep.cpu().numpy(), "count": cnt.cpu().numpy(), "best": best.cpu().numpy(),
                "choice": ch.cpu().numpy()}
    finally:
        ctx.free(did)


def oracle_choices(ref, kind):
    """Per-round pole choices implied by the oracle's own round minima."""
    rm, ra = ref["round_min"], ref["round_arg"]
    out = np.full(rm.shape, -1, np.int32)
    for q in range(rm.shape[0]):
        dmin = 1.0
        for l in range(rm.shape[1]):
            if rm[q, l] < dmin:
                dmin = rm[q, l]
                out[q, l] = ra[q, l]
    return out


def assert_hd_exact(g, ref):
    np.testing.assert_array_equal(g["count"], ref["count"])
    np.testing.assert_array_equal(g["depth"], ref["depth"])
    np.testing.assert_array_equal(g["best"], ref["best"])


def assert_follow(g, X, Z, kind, k, r, alpha, seed, qidx=None, tol=TOL):
    ref = oracle.rrs(X, Z, kind, k, r, alpha, seed, qidx=qidx, follow=g["choice"])
    rf, rm = ref["round_at_follow"], ref["round_min"]
    taken = g["choice"] >= 0
    # every pole the GPU took is a round minimum of the oracle's depths, within tol
    assert np.all(rf[taken] <= rm[taken] * (1 + tol) + 1e-300), "GPU took a direction that is not a round minimum"
    # rounds where the GPU kept the pole: the oracle's round minimum does not beat D_min by more than tol
    for q in range(Z.shape[0]):
        dmin = 1.0
        for l in range(r):
            if taken[q, l]:
                dmin = rf[q, l]
            else:
                assert rm[q, l] >= dmin * (1 - tol), (q, l)
    rel = np.abs(g["depth"] - ref["depth"]) / np.maximum(ref["depth"], 1e-300)
    assert np.max(rel) <= tol, f"max relative error {np.max(rel):.3e}"
    np.testing.assert_array_equal(g["best"], ref["best"])
    return ref


# ------------------------------------------------------------------------------------------
# direction stream
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("d,m,rnd,alpha", [(1, 37, 1, 0.5), (2, 100, 1, 0.5), (2, 100, 7, 0.5), (10, 50, 1, 0.7),
                                           (10, 50, 20, 0.7), (50, 130, 3, 0.9), (97, 64, 10, 0.9)])
def test_direction_stream_bit_exact(ctx, d, m, rnd, alpha):
    rng = np.random.default_rng(d * 100 + rnd)
    pole = rng.standard_normal(d).astype(np.float32)
    pole /= np.float32(np.linalg.norm(pole))
    for seed, q in ((0, 0), (12345, 77), (2 ** 63 + 5, 4096)):
        U = torch.empty((m, d), dtype=torch.float32, device="cuda")
        pt = torch.from_numpy(pole).cuda()
        rrs.rrs_debug_directions(ctx.handle, seed, q, rnd, m, d, alpha, pt, U)
        ref = oracle.directions(seed, q, rnd - 1, m, d, alpha, pole)
        got = U.cpu().numpy()
        assert np.array_equal(got.view(np.uint32), ref.view(np.uint32)), \
            f"{int(np.sum(got.view(np.uint32) != ref.view(np.uint32)))} differing words"


# ------------------------------------------------------------------------------------------
# halfspace depth: exact
# ------------------------------------------------------------------------------------------

def test_c1_halfspace_full_bit_exact(ctx):
    Pr = workloads.c1()
    g = gpu_rrs(ctx, Pr.X, Pr.Z, H, Pr.k, Pr.r, Pr.alpha, Pr.seed)
    ref = oracle.rrs(Pr.X, Pr.Z, H, Pr.k, Pr.r, Pr.alpha, Pr.seed, rounds=True)
    assert_hd_exact(g, ref)
    np.testing.assert_array_equal(g["choice"], oracle_choices(ref, H))


@pytest.mark.parametrize("n,d,dtype", [(1, 3, np.float32), (2, 1, np.float64), (63, 5, np.float32),
                                       (1037, 50, np.float32), (2500, 17, np.float64), (700, 100, np.float32)])
def test_halfspace_bit_exact_shapes(ctx, n, d, dtype):
    X, Z = workloads.gaussian_cloud(n + d, n, d, 7, dtype=dtype, zscale=1.2)
    Z[0] = X[0]   # a query on a data point: exact ties on every direction
    g = gpu_rrs(ctx, X, Z, H, 130, 3, 0.6, seed=5)
    ref = oracle.rrs(X, Z, H, 130, 3, 0.6, 5, rounds=True)
    assert_hd_exact(g, ref)
    np.testing.assert_array_equal(g["choice"], oracle_choices(ref, H))


def test_halfspace_integer_grid_ties(ctx):
    # many exact ties u'(x - z) = 0 are impossible for random u, but duplicates and z = x_i are not
    rng = np.random.default_rng(3)
    X = rng.integers(-3, 4, size=(400, 3)).astype(np.float32)
    Z = np.concatenate([X[:5], rng.integers(-3, 4, size=(5, 3)).astype(np.float32)])
    g = gpu_rrs(ctx, X, Z, H, 200, 4, 0.5, seed=1)
    ref = oracle.rrs(X, Z, H, 200, 4, 0.5, 1)
    assert_hd_exact(g, ref)


def test_halfspace_round_counts_and_band(ctx):
    # per-direction counts for caller-supplied directions, several tiles and a ragged tail
    X, Z = workloads.gaussian_cloud(8, 1000 + 37, 6, 3, dtype=np.float32)
    m = 70
    U = np.stack([oracle.directions(3, q, 0, m, 6, 0.5) for q in range(3)])
    did = ctx.register(torch.from_numpy(X).cuda())
    dep = torch.empty((3, m), dtype=torch.float64, device="cuda")
    cnt = torch.empty((3, m), dtype=torch.int64, device="cuda")
    band = torch.zeros(3, dtype=torch.int64, device="cuda")
    rrs.rrs_debug_round_depths(ctx.handle, did, torch.from_numpy(Z).cuda(), 3, rrs.RRS_F32, H, m,
                               torch.from_numpy(U).cuda(), rrs.RRS_PREC_FP32_SIMT, dep, cnt, band)
    ctx.free(did)
    for q in range(3):
        for j in range(m):
            d_ref, c_ref = oracle.univariate(H, X, Z[q], U[q, j])
            assert cnt[q, j].item() == c_ref
            assert dep[q, j].item() == d_ref


def test_halfspace_far_point_and_centre(ctx):
    rng = np.random.default_rng(4)
    half = rng.standard_normal((300, 4)).astype(np.float32)
    X = np.concatenate([half, -half])
    Z = np.array([[0, 0, 0, 0], [40, 40, 40, 40]], dtype=np.float32)
    g = gpu_rrs(ctx, X, Z, H, 100, 2, 0.5)
    assert g["count"][0] == 300 and g["count"][1] == 0


# ------------------------------------------------------------------------------------------
# projection / asymmetric projection depth: follow mode, 1e-5 relative
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("kind", [P, AP])
def test_c2_shape_small_follow(ctx, kind):
    Pr = workloads.c2(n=2000, nq=40, kind=kind)
    g = gpu_rrs(ctx, Pr.X, Pr.Z, kind, 200, 5, Pr.alpha, 0)
    assert_follow(g, Pr.X, Pr.Z, kind, 200, 5, Pr.alpha, 0)


@pytest.mark.parametrize("kind", [P, AP])
@pytest.mark.parametrize("n,d", [(1, 2), (2, 3), (2, 10), (3, 1), (3, 5), (4, 6), (64, 4), (1001, 10), (4096, 7),
                                 (20000, 3)])
def test_projection_depth_shapes(ctx, kind, n, d):
    # With d >= n - 1 RRS steers u towards directions where two projections coincide and the MAD
    # (or MAD_+) goes to 0; the selection picks the points on FP32 keys and the depth is formed from
    # their FP64 projections, so the small spread keeps its relative accuracy.
    X, Z = workloads.gaussian_cloud(n * 3 + d, n, d, 6, dtype=np.float32)
    Z[0] = X[0]
    g = gpu_rrs(ctx, X, Z, kind, 60, 3, 0.5, seed=2)
    assert_follow(g, X, Z, kind, 60, 3, 0.5, 2)


@pytest.mark.parametrize("kind", [P, AP])
@pytest.mark.parametrize("n,d", [(3000, 17), (2500, 50), (1200, 150)])
def test_projection_depth_large_d(ctx, kind, n, d):
    # d > 16: keys formed by the tiled GEMM and read by the selection kernel
    X, Z = workloads.gaussian_cloud(n + d, n, d, 6, dtype=np.float32, zscale=0.8)
    g = gpu_rrs(ctx, X, Z, kind, 240, 3, 0.8, 5)
    assert_follow(g, X, Z, kind, 240, 3, 0.8, 5)


@pytest.mark.parametrize("kind", [P, AP])
def test_projection_round_depths(ctx, kind):
    X, Z = workloads.gaussian_cloud(9, 3001, 10, 2, dtype=np.float32)
    m = 50
    U = np.stack([oracle.directions(1, q, 0, m, 10, 0.5) for q in range(2)])
    did = ctx.register(torch.from_numpy(X).cuda())
    dep = torch.empty((2, m), dtype=torch.float64, device="cuda")
    rrs.rrs_debug_round_depths(ctx.handle, did, torch.from_numpy(Z).cuda(), 2, rrs.RRS_F32, kind, m,
                               torch.from_numpy(U).cuda(), rrs.RRS_PREC_FP32_SIMT, dep)
    ctx.free(did)
    got = dep.cpu().numpy()
    for q in range(2):
        ref = np.array([oracle.univariate(kind, X, Z[q], U[q, j])[0] for j in range(m)])
        np.testing.assert_allclose(got[q], ref, rtol=TOL)


def test_projection_degenerate_constant_cloud(ctx):
    X = np.ones((50, 3), np.float32)
    Z = np.array([[1, 1, 1], [1, 2, 1]], np.float32)
    for kind in (P, AP):
        g = gpu_rrs(ctx, X, Z, kind, 40, 2, 0.5)
        ref = oracle.rrs(X, Z, kind, 40, 2, 0.5)
        np.testing.assert_array_equal(g["depth"], ref["depth"])


# ------------------------------------------------------------------------------------------
# boundary behaviour
# ------------------------------------------------------------------------------------------

def test_host_buffers_match_device_buffers(ctx):
    X, Z = workloads.gaussian_cloud(21, 500, 4, 5, dtype=np.float32)
    a = gpu_rrs(ctx, X, Z, H, 90, 3, 0.5, seed=4, on_device=True)
    did = rrs.rrs_register_dataset(ctx.handle, X, X.shape[0], 4, rrs.RRS_F32, False)
    dep = np.zeros(5)
    cnt = np.zeros(5, np.int64)
    best = np.zeros(5, np.int32)
    rrs.rrs_depth(ctx.handle, did, Z, 5, rrs.RRS_F32, False, H, 90, 3, 0.5, 4, rrs.RRS_PREC_FP32_SIMT, dep, cnt,
                  best, None, False, None)
    rrs.rrs_free(ctx.handle, did)
    np.testing.assert_array_equal(dep, a["depth"])
    np.testing.assert_array_equal(cnt, a["count"])
    np.testing.assert_array_equal(best, a["best"])


def test_errors_are_reported_not_raised_on_device(ctx):
    X = np.zeros((10, 2), np.float32)
    did = rrs.rrs_register_dataset(ctx.handle, X, 10, 2, rrs.RRS_F32, False)
    dep = np.zeros(1)
    Z = np.zeros((1, 2), np.float32)
    for bad in [dict(k=5, r=10), dict(k=10, r=2, alpha=1.5), dict(k=10, r=2, alpha=0.0)]:
        with pytest.raises(rrs.RRSError) as e:
            rrs.rrs_depth(ctx.handle, did, Z, 1, rrs.RRS_F32, False, H, bad["k"], bad["r"], bad.get("alpha", 0.5), 0,
                          0, dep, None, None, None, False, None)
        assert e.value.status == rrs.RRS_ERR_INVALID_ARG
    with pytest.raises(rrs.RRSError) as e:
        rrs.rrs_depth(ctx.handle, did + 999, Z, 1, rrs.RRS_F32, False, H, 10, 2, 0.5, 0, 0, dep, None, None, None,
                      False, None)
    assert e.value.status == rrs.RRS_ERR_NOT_FOUND
    Zbad = np.array([[np.nan, 0]], np.float32)
    with pytest.raises(rrs.RRSError) as e:
        rrs.rrs_depth(ctx.handle, did, Zbad, 1, rrs.RRS_F32, False, H, 10, 2, 0.5, 0, 0, dep, None, None, None,
                      False, None)
    assert e.value.status == rrs.RRS_ERR_INVALID_ARG
    Xbad = np.array([[np.inf, 0]], np.float32)
    with pytest.raises(rrs.RRSError) as e:
        rrs.rrs_register_dataset(ctx.handle, Xbad, 1, 2, rrs.RRS_F32, False)
    assert e.value.status == rrs.RRS_ERR_INVALID_ARG
    rrs.rrs_free(ctx.handle, did)
    with pytest.raises(rrs.RRSError):
        rrs.rrs_free(ctx.handle, did)   # double free is an error, not a crash
    # the context still works after the errors
    X2, Z2 = workloads.gaussian_cloud(1, 50, 2, 2, dtype=np.float32)
    g = gpu_rrs(ctx, X2, Z2, H, 20, 2, 0.5)
    assert np.all(g["count"] >= 0)


@pytest.mark.parametrize("kind", [P, AP])
def test_projection_depth_either_side_of_the_shared_memory_limit(ctx, kind):
    # one direction's 55,000 FP32 keys still fit a CTA's 227 KB of shared memory; 56,000 do not, and
    # there the keys live in device memory and every selection pass reads them: both sides against the oracle
    for seed_data, n in ((77, 55_000), (78, 56_000)):
        X, Z = workloads.gaussian_cloud(seed_data, n, 4, 3, dtype=np.float32)
        g = gpu_rrs(ctx, X, Z, kind, 30, 2, 0.7, 2)
        assert_follow(g, X, Z, kind, 30, 2, 0.7, 2)
    X, Z = workloads.gaussian_cloud(79, 500, 4, 3, dtype=np.float32)
    g2 = gpu_rrs(ctx, X, Z, kind, 30, 2, 0.7, 2)   # a resident-key dataset right after: no state carried over
    assert_follow(g2, X, Z, kind, 30, 2, 0.7, 2)


@pytest.mark.parametrize("kind", [P, AP])
@pytest.mark.parametrize("n,d", [(70_001, 10), (65_000, 20), (120_000, 3)])
def test_projection_depth_keys_outside_shared_memory(ctx, kind, n, d):
    # keys outside shared memory, formed once by the keys kernels and read by every selection pass: odd n
    # (ragged tail of the four-wide scans), d > 16 (tiled GEMM keys) and twice the shared-memory limit
    X, Z = workloads.gaussian_cloud(90 + d, n, d, 2, dtype=np.float32)
    g = gpu_rrs(ctx, X, Z, kind, 24, 2, 0.7, 5)
    assert_follow(g, X, Z, kind, 24, 2, 0.7, 5)


@pytest.mark.parametrize("kind", [P, AP])
@pytest.mark.parametrize("n", [20_000, 60_000])
def test_projection_depth_heavy_tails(ctx, kind, n):
    # multivariate t with one degree of freedom: bucket ranges from the covariance are far too wide, so
    # selections go through the iterated-bucket fallback, with keys in shared memory (n = 20,000) and in
    # device memory (n = 60,000)
    X, Z, _ = workloads.ranking_cloud(300 + n % 7, n, 5, 1.0, 3)
    g = gpu_rrs(ctx, X, Z, kind, 24, 2, 0.7, 8)
    assert_follow(g, X, Z, kind, 24, 2, 0.7, 8)


@pytest.mark.parametrize("kind", [P, AP])
@pytest.mark.parametrize("n", [20_000, 60_000])
def test_projection_depth_lattice_ties(ctx, kind, n):
    # 343 distinct rows repeated ~n/343 times: long runs of equal keys around the median and the MAD,
    # beyond the gather buffer, resolved exactly
    rng = np.random.default_rng(n)
    X = rng.integers(-3, 4, size=(n, 3)).astype(np.float32)
    Z = np.array([[0, 0, 0], [1, -1, 2], [3, 3, 3]], np.float32)
    g = gpu_rrs(ctx, X, Z, kind, 24, 2, 0.7, 9)
    assert_follow(g, X, Z, kind, 24, 2, 0.7, 9)


def test_halfspace_beyond_the_direction_stage(ctx):
    # d = 200: directions wider than the generator's shared-memory stage are built in place in device
    # memory; counts, depths and best indices still bit-exact
    X, Z = workloads.gaussian_cloud(41, 300, 200, 3, dtype=np.float32)
    g = gpu_rrs(ctx, X, Z, H, 40, 2, 0.6, 3)
    assert_hd_exact(g, oracle.rrs(X, Z, H, 40, 2, 0.6, 3))


def test_zero_queries_is_a_no_op(ctx):
    X = np.ones((4, 2), np.float32)
    did = rrs.rrs_register_dataset(ctx.handle, X, 4, 2, rrs.RRS_F32, False)
    rrs.rrs_depth(ctx.handle, did, None, 0, rrs.RRS_F32, False, H, 10, 2, 0.5, 0, 0, None, None, None, None, False,
                  None)
    rrs.rrs_free(ctx.handle, did)


def test_budget_is_enforced():
    c = rrs.Context(0, hbm_budget_bytes=4096)
    X = np.zeros((10000, 8), np.float32)
    with pytest.raises(rrs.RRSError) as e:
        c.register(torch.from_numpy(X))
    assert e.value.status == rrs.RRS_ERR_BUDGET
    c.close()


def test_bounded_wait_reports_timeout_and_context_survives(ctx):
    # a device wait on a barrier nothing completes gives up (about 1 ms of SM clock) and reports it
    with pytest.raises(rrs.RRSError) as e:
        rrs.rrs_debug_wait_timeout(ctx.handle, 2_000_000)
    assert e.value.status == rrs.RRS_ERR_TIMEOUT
    X, Z = workloads.gaussian_cloud(3, 100, 3, 2, dtype=np.float32)
    g = gpu_rrs(ctx, X, Z, H, 30, 2, 0.5)
    ref = oracle.rrs(X, Z, H, 30, 2, 0.5)
    np.testing.assert_array_equal(g["count"], ref["count"])


@pytest.mark.parametrize("kind", [P, AP])
def test_autotuned_group_does_not_change_results(ctx, kind):
    X, Z = workloads.gaussian_cloud(31, 5000, 10, 30, dtype=np.float32)
    did = ctx.register(torch.from_numpy(X).cuda())
    Zt = torch.from_numpy(Z).cuda()
    before = ctx.depth(did, Zt, kind, 100, 4, 0.7, 3)[0].cpu().numpy()
    g = rrs.rrs_autotune(ctx.handle, did, kind, 100, 4)
    assert g in (1, 2, 4, rrs.RRS_SELECT_WARP, rrs.RRS_SELECT_STREAM)
    after = ctx.depth(did, Zt, kind, 100, 4, 0.7, 3)[0].cpu().numpy()
    ctx.free(did)
    np.testing.assert_array_equal(before, after)


@pytest.mark.parametrize("kind", [P, AP])
@pytest.mark.parametrize("n,d,m", [(3001, 10, 50), (777, 5, 37), (12288, 16, 25), (9000, 3, 13), (40, 7, 24),
                                   (2, 4, 12)])
def test_every_selection_kernel_selects_the_same_points(ctx, kind, n, d, m):
    # the warp-per-direction kernel (keys re-formed at every pass), the shared-memory kernels with 1, 2 or 4
    # directions per CTA and the streamed-keys kernel rank the same FP32 keys by (value, index) and form the
    # depth from the same FP64 projections: bit-identical depths and per-round choices whatever kernel runs
    X, Z = workloads.gaussian_cloud(n + 7 * d + m, n, d, 9, dtype=np.float32)
    did = ctx.register(torch.from_numpy(X).cuda())
    Zt = torch.from_numpy(Z).cuda()
    k, r = 3 * m, 3
    out = {}
    for choice in (0, 1, 2, 4, rrs.RRS_SELECT_WARP, rrs.RRS_SELECT_STREAM):
        rrs.rrs_select_kernel(ctx.handle, did, k, r, choice)
        dep, _, best, ch = ctx.depth(did, Zt, kind, k, r, 0.6, 4, rounds=True)
        out[choice] = (dep.cpu().numpy(), best.cpu().numpy(), ch.cpu().numpy())
    rrs.rrs_select_kernel(ctx.handle, did, k, r, 0)
    ctx.free(did)
    for choice, (dep, best, ch) in out.items():
        np.testing.assert_array_equal(dep, out[0][0], err_msg=f"choice {choice}")
        np.testing.assert_array_equal(best, out[0][1], err_msg=f"choice {choice}")
        np.testing.assert_array_equal(ch, out[0][2], err_msg=f"choice {choice}")
    g = {"depth": out[0][0], "best": out[0][1], "choice": out[0][2], "count": None}
    assert_follow(g, X, Z, kind, k, r, 0.6, 4)


def test_kernel_choices_reject_unknown_values(ctx):
    X, _ = workloads.gaussian_cloud(5, 100, 4, 1, dtype=np.float32)
    did = ctx.register(torch.from_numpy(X).cuda())
    for bad in (3, 8, -1, 1000):
        with pytest.raises(rrs.RRSError) as e:
            rrs.rrs_select_kernel(ctx.handle, did, 100, 4, bad)
        assert e.value.status == rrs.RRS_ERR_INVALID_ARG
    for bad in (64, 512, -1):
        with pytest.raises(rrs.RRSError) as e:
            rrs.rrs_select_tc_tile(ctx.handle, did, bad)
        assert e.value.status == rrs.RRS_ERR_INVALID_ARG
    with pytest.raises(rrs.RRSError) as e:
        rrs.rrs_select_kernel(ctx.handle, 123456, 100, 4, 2)
    assert e.value.status == rrs.RRS_ERR_NOT_FOUND
    ctx.free(did)
