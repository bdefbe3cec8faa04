"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test names what fixes the expected value: an independent library
implementation, a closed form worked out by hand, exact rational arithmetic,
an independent exact algorithm, a limit theorem or an exact invariance.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import exact2d
import workloads

H, P, AP = 0, 1, 2


# --------------------------------------------------------------------------
# Philox4x32-10 against Triton's independent implementation (CPU interpreter)
# --------------------------------------------------------------------------

def _triton_philox(counters, seed):
    os.environ["TRITON_INTERPRET"] = "1"
    try:
        import torch
        import triton
        import triton.language as tl
    except Exception as e:  # pragma: no cover
        pytest.skip(f"triton interpreter unavailable: {e}")

    @triton.jit
    def _k(out_ptr, seed, c0p, c1p, c2p, c3p, N: tl.constexpr):
        o = tl.arange(0, N)
        a, b, c, d = tl.philox(seed, tl.load(c0p + o), tl.load(c1p + o), tl.load(c2p + o),
                               tl.load(c3p + o), 10)
        tl.store(out_ptr + o * 4 + 0, a)
        tl.store(out_ptr + o * 4 + 1, b)
        tl.store(out_ptr + o * 4 + 2, c)
        tl.store(out_ptr + o * 4 + 3, d)

    C = np.asarray(counters, dtype=np.uint32)
    N = C.shape[0]
    cols = [torch.from_numpy(C[:, i].astype(np.int64).astype(np.uint32).view(np.int32).copy())
            for i in range(4)]
    out = torch.zeros(N * 4, dtype=torch.int32)
    _k[(1,)](out, seed, cols[0], cols[1], cols[2], cols[3], N)
    return out.numpy().view(np.uint32).reshape(N, 4)


def test_philox_matches_triton_interpreter():
    rng = np.random.default_rng(11)
    C = rng.integers(0, 2 ** 32, size=(16, 4), dtype=np.uint64).astype(np.uint32)
    C[0] = 0
    C[1] = [0xFFFFFFFF] * 4
    C[2] = [5, 17, 3, 99]  # a (b, j, round, q) counter of the direction stream
    for seed in (0, 1, 0x123456789ABCDEF, 2 ** 64 - 1):
        ref = _triton_philox(C, seed)
        key = [seed & 0xFFFFFFFF, seed >> 32]
        got = np.stack([oracle.philox4x32_10(c, key) for c in C])
        np.testing.assert_array_equal(got, ref)


# --------------------------------------------------------------------------
# FP32 transcendentals of the direction stream against FP64 libm
# --------------------------------------------------------------------------

def _ulp32(v):
    return np.spacing(np.abs(np.float32(v))).astype(np.float64)


def test_logf_accuracy():
    rng = np.random.default_rng(0)
    w = rng.integers(0, 2 ** 32, size=4000, dtype=np.uint64)
    U = ((2 * (w >> 9) + 1).astype(np.float64) * 2.0 ** -24).astype(np.float32)
    U = np.concatenate([U, np.float32([2.0 ** -24, 0.5, 0.70710677, 0.7071068, 1.0 - 2.0 ** -24])])
    for u in U:
        got = float(oracle.logf(u))
        ref = math.log(float(u))
        assert abs(got - ref) <= 4 * _ulp32(ref) + 1e-45, (u, got, ref)


def test_sincos_quarter_turn_accuracy():
    a = np.concatenate([np.linspace(0, 4, 2001, endpoint=False), [0.5, 1.5, 2.5, 3.5, 1e-6, 3.9999998]])
    for v in a.astype(np.float32):
        s, c = oracle.sincos_qturn(v)
        ang = math.pi / 2 * float(v)
        assert abs(float(s) - math.sin(ang)) <= 3e-7, v
        assert abs(float(c) - math.cos(ang)) <= 3e-7, v
        assert abs(float(s) ** 2 + float(c) ** 2 - 1.0) < 1e-6


# --------------------------------------------------------------------------
# Direction stream: uniform on the sphere (Alg. S1) and inside the cap (Alg. S4)
# --------------------------------------------------------------------------

def test_round1_directions_uniform_on_sphere():
    d, m = 5, 4000
    U = np.concatenate([oracle.directions(7, q, 0, m, d, 0.5) for q in range(5)]).astype(np.float64)
    assert np.all(np.abs(np.linalg.norm(U, axis=1) - 1.0) < 1e-6)
    # moments of the uniform law on S^{d-1}: E u = 0, E u u^T = I/d, E u_1^4 = 3/(d(d+2))
    N = U.shape[0]
    assert np.all(np.abs(U.mean(axis=0)) < 4.5 / math.sqrt(N * d))
    C = U.T @ U / N
    assert np.max(np.abs(C - np.eye(d) / d)) < 0.01
    m4 = np.mean(U[:, 0] ** 4)
    assert abs(m4 - 3.0 / (d * (d + 2))) < 0.01
    # both hemispheres are used (the first round is the whole sphere)
    assert 0.45 < np.mean(U[:, 0] > 0) < 0.55


def test_cap_directions_follow_the_pole():
    d = 6
    rng = np.random.default_rng(3)
    pole = rng.standard_normal(d).astype(np.float32)
    pole /= np.float32(np.linalg.norm(pole))
    for alpha, rnd in ((0.5, 1), (0.5, 3), (0.9, 10), (0.7, 19)):
        cap = math.pi / 2 * alpha ** rnd
        U = oracle.directions(1, 0, rnd, 3000, d, alpha, pole).astype(np.float64)
        nrm = np.linalg.norm(U, axis=1)
        assert np.all(np.abs(nrm - 1.0) < 2e-6)
        ang = np.arccos(np.clip(U @ pole.astype(np.float64) / nrm, -1, 1))
        assert ang.max() <= cap * (1 + 1e-3) + 2e-6
        # theta = V * cap with V uniform: the angle is uniform in [0, cap]
        if cap > 1e-2:
            a = np.sort(ang / cap)
            ks = np.max(np.abs(a - np.arange(1, a.size + 1) / a.size))
            assert ks < 1.63 / math.sqrt(a.size) + 2e-3, (alpha, rnd, ks)
        # the component orthogonal to the pole is isotropic: its mean is ~0
        orth = U - np.outer(U @ pole, pole)
        orth /= np.linalg.norm(orth, axis=1, keepdims=True)
        assert np.all(np.abs(orth.mean(axis=0)) < 0.08)


def test_cap_direction_at_pole_e1_is_identity_map():
    d = 4
    e1 = np.zeros(d, np.float32)
    e1[0] = 1
    U = oracle.directions(5, 2, 4, 200, d, 0.5, e1).astype(np.float64)
    cap = math.pi / 2 * 0.5 ** 4
    assert np.all(U[:, 0] >= math.cos(cap) - 1e-6)


def test_d1_directions_are_signs():
    U = oracle.directions(0, 0, 0, 1000, 1, 0.5)
    assert np.all(np.abs(np.abs(U) - 1.0) < 1e-6)
    assert 400 < int((U > 0).sum()) < 600


# --------------------------------------------------------------------------
# Exact halfspace signs against rational arithmetic
# --------------------------------------------------------------------------

def test_exact_sign_matches_fractions_on_near_ties():
    rng = np.random.default_rng(5)
    for trial in range(400):
        d = int(rng.integers(1, 7))
        u = rng.standard_normal(d).astype(np.float32)
        z = rng.standard_normal(d)
        if trial % 4 == 0:
            x = z.copy()                                  # exact tie: x = z
        elif trial % 4 == 1 and d >= 2:
            # x - z orthogonal to u up to one FP64 rounding: a near tie
            w = rng.standard_normal(d)
            w -= (w @ u.astype(np.float64)) / float(u.astype(np.float64) @ u.astype(np.float64)) * u
            x = z + w
        elif trial % 4 == 2:
            x = z + rng.standard_normal(d) * 1e-15       # tiny offsets
        else:
            x = rng.standard_normal(d) * 10.0 ** rng.integers(-3, 4)
        ref = exact2d.sign_fraction(u, x, z)
        assert oracle.exact_sign(u, x, z) == ref, (trial, u, x, z)


def test_exact_sign_integer_hyperplane():
    # u = (1, 2), x - z = (2, -1): exactly orthogonal with large offsets
    u = np.float32([1.0, 2.0])
    z = np.array([1e8 + 0.5, -3e-8])
    x = z + np.array([2.0, -1.0])
    assert oracle.exact_sign(u, x, z) == exact2d.sign_fraction(u, x, z)


# --------------------------------------------------------------------------
# Univariate depths: exact arithmetic, closed forms worked by hand, invariances
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind", [H, P, AP])
def test_univariate_matches_exact_rationals(kind):
    rng = np.random.default_rng(kind + 10)
    for trial in range(60):
        n = int(rng.integers(1, 9))
        d = int(rng.integers(1, 4))
        X = rng.integers(-3, 4, size=(n, d)).astype(np.float64) * 0.5  # ties are frequent
        if trial % 3 == 0:
            X = rng.standard_normal((n, d))
        z = X[rng.integers(0, n)] if trial % 2 else rng.standard_normal(d)
        u = rng.standard_normal(d).astype(np.float32)
        got, cnt = oracle.univariate(kind, X, z, u)
        ref = exact2d.univariate_fraction(kind, X, z, u)
        assert abs(got - float(ref)) <= 1e-12 * max(1.0, float(ref)), (kind, trial, got, ref)
        if kind == H:
            assert cnt == ref * n


def test_projection_depth_closed_form_arithmetic_sequence():
    # X = {1..n}, n = 2k+1: med = k+1; |x - med| = 0,1,1,...,k,k -> MAD = ceil(k/2);
    # the positive deviations are 1..k -> MAD_+ = (k+1)/2.
    for k in (2, 3, 7, 10):
        n = 2 * k + 1
        X = np.arange(1, n + 1, dtype=np.float64)[:, None]
        med, mad, madp = k + 1, math.ceil(k / 2), (k + 1) / 2
        for zv in (0.25, med, med + 1.5, n + 3.0):
            z = np.array([zv])
            dp, _ = oracle.univariate(P, X, z, np.float32([1.0]))
            assert dp == pytest.approx(1.0 / (1.0 + abs(zv - med) / mad), rel=1e-15)
            dap, _ = oracle.univariate(AP, X, z, np.float32([1.0]))
            assert dap == pytest.approx(1.0 / (1.0 + max(zv - med, 0.0) / madp), rel=1e-15)
            dh, c = oracle.univariate(H, X, z, np.float32([1.0]))
            le = int(np.sum(X[:, 0] <= zv))
            ge = int(np.sum(X[:, 0] >= zv))
            assert c == min(le, ge)


def test_even_count_median_and_degenerate_mad():
    X = np.array([[1.0], [2.0], [4.0], [8.0]])  # med = 3, |dev| = 2,1,1,5 -> MAD = 1.5
    dp, _ = oracle.univariate(P, X, np.array([6.0]), np.float32([1.0]))
    assert dp == pytest.approx(1.0 / (1.0 + 3.0 / 1.5), rel=1e-15)
    # positive deviations {1, 5} -> MAD_+ = 3
    dap, _ = oracle.univariate(AP, X, np.array([6.0]), np.float32([1.0]))
    assert dap == pytest.approx(1.0 / (1.0 + 3.0 / 3.0), rel=1e-15)
    # all points equal: MAD = 0 -> depth 1 at the point, 0 elsewhere
    X0 = np.ones((5, 2))
    assert oracle.univariate(P, X0, np.ones(2), np.float32([0.6, 0.8]))[0] == 1.0
    assert oracle.univariate(P, X0, np.array([1.0, 2.0]), np.float32([0.6, 0.8]))[0] == 0.0
    assert oracle.univariate(AP, X0, np.array([0.0, 0.0]), np.float32([0.6, 0.8]))[0] == 1.0


@pytest.mark.parametrize("kind", [H, P, AP])
def test_univariate_exact_invariances(kind):
    rng = np.random.default_rng(20 + kind)
    X = rng.standard_normal((301, 4))
    z = rng.standard_normal(4)
    u = rng.standard_normal(4).astype(np.float32)
    base = oracle.univariate(kind, X, z, u)
    for s in (-3, 5):  # power-of-two scaling is exact
        assert oracle.univariate(kind, X * 2.0 ** s, z * 2.0 ** s, u) == base
    perm = rng.permutation(X.shape[0])
    assert oracle.univariate(kind, X[perm], z, u) == base
    # negating data, query and direction leaves every projection unchanged
    assert oracle.univariate(kind, -X, -z, -u) == base
    # positive scaling of the direction by a power of two
    assert oracle.univariate(kind, X, z, u * np.float32(4.0)) == base


@pytest.mark.parametrize("kind", [H, P, AP])
def test_rrs_translation_invariance_exact(kind):
    # depth is translation invariant (Sec. 2: every univariate depth sees y - y_z or y - med).  With small
    # integer data, an integer shift and FP32 directions every FP64 product and sum is exact, so the whole
    # search (same directions, same decisions) must return identical results
    rng = np.random.default_rng(30 + kind)
    X = rng.integers(-20, 21, size=(257, 3)).astype(np.float64)
    Z = rng.integers(-10, 11, size=(6, 3)).astype(np.float64)
    c = np.array([37.0, -12.0, 5.0])
    a = oracle.rrs(X, Z, kind, 90, 3, 0.6, 4)
    b = oracle.rrs(X + c, Z + c, kind, 90, 3, 0.6, 4)
    np.testing.assert_array_equal(a["depth"], b["depth"])
    np.testing.assert_array_equal(a["count"], b["count"])
    np.testing.assert_array_equal(a["best"], b["best"])


def test_asymmetric_depth_is_not_symmetric():
    # D_AP(z|X along u) != D_AP(-z|-X along u) in general (Supp. A symmetry fails)
    X = np.array([[0.0], [1.0], [1.0], [10.0], [11.0]])
    z = np.array([12.0])
    a = oracle.univariate(AP, X, z, np.float32([1.0]))[0]
    b = oracle.univariate(AP, -X, -z, np.float32([1.0]))[0]
    assert a != b


# --------------------------------------------------------------------------
# Whole RRS runs
# --------------------------------------------------------------------------

def test_rrs_never_below_exact_2d_halfspace_depth():
    Pr = workloads.c1()
    Zs = Pr.Z[:40]
    ex = exact2d.halfspace_depth_2d(Pr.X, Zs)
    out = oracle.rrs(Pr.X, Zs, H, Pr.k, Pr.r, Pr.alpha, Pr.seed)
    assert np.all(out["count"] >= ex)           # the Corollary of Sec. 2
    assert np.mean(out["count"] == ex) >= 0.8   # 1,000 directions in d=2 nearly always hit
    assert np.max(out["count"] - ex) <= 3
    np.testing.assert_allclose(out["depth"], out["count"] / Pr.n)


def test_rrs_tiny_brute_force_2d():
    rng = np.random.default_rng(9)
    for trial in range(20):
        n = int(rng.integers(1, 9))
        X = rng.integers(-4, 5, size=(n, 2)).astype(np.float64)
        Z = rng.integers(-4, 5, size=(3, 2)).astype(np.float64)
        ex = exact2d.halfspace_depth_2d(X, Z)
        out = oracle.rrs(X, Z, H, 400, 4, 0.5, trial)
        assert np.all(out["count"] >= ex)
        assert np.all(out["count"] <= n)


def test_rrs_d1_closed_forms():
    X = np.arange(1, 16, dtype=np.float64)[:, None]   # n = 15, k = 7: med 8, MAD 4, MAD_+ 4, MAD_- 4
    Z = np.array([[0.5], [8.0], [9.5], [20.0]])
    h = oracle.rrs(X, Z, H, 200, 4, 0.5)
    np.testing.assert_array_equal(h["count"], [0, 8, 6, 0])
    p = oracle.rrs(X, Z, P, 200, 4, 0.5)
    np.testing.assert_allclose(p["depth"], [1 / (1 + 7.5 / 4), 1.0, 1 / (1 + 1.5 / 4), 1 / (1 + 12 / 4)],
                               rtol=1e-14)
    a = oracle.rrs(X, Z, AP, 200, 4, 0.5)   # both signs of u appear: min over both tails
    np.testing.assert_allclose(a["depth"], [1 / (1 + 7.5 / 4), 1.0, 1 / (1 + 1.5 / 4), 1 / (1 + 12 / 4)],
                               rtol=1e-14)


def test_rrs_centrally_symmetric_cloud():
    rng = np.random.default_rng(4)
    half = rng.standard_normal((200, 3))
    X = np.concatenate([half, -half])
    z = np.zeros((1, 3))
    h = oracle.rrs(X, z, H, 300, 3, 0.5)
    assert h["count"][0] == 200                 # every halfspace through 0 holds exactly half
    p = oracle.rrs(X, z, P, 300, 3, 0.5)
    assert p["depth"][0] == 1.0                 # med = 0 along every direction


def test_rrs_far_point_has_zero_halfspace_depth():
    X, Z = workloads.gaussian_cloud(12, 500, 5, 3)
    Z = Z + 50.0
    h = oracle.rrs(X, Z, H, 500, 5, 0.5)
    assert np.all(h["count"] == 0)


@pytest.mark.slow
def test_rrs_gaussian_limits():
    # X ~ N(0, I_3): PD(z) = AP(z) -> 1/(1 + |z|/q75), HD(z) -> 1 - Phi(|z|)
    from scipy.stats import norm
    q75 = norm.ppf(0.75)
    X, _ = workloads.gaussian_cloud(13, 20000, 3, 1)
    radii = np.array([0.0, 0.5, 1.0, 2.0])
    rng = np.random.default_rng(1)
    dirs = rng.standard_normal((radii.size, 3))
    Z = dirs / np.linalg.norm(dirs, axis=1, keepdims=True) * radii[:, None]
    tol = 3.0 / math.sqrt(X.shape[0]) + 0.01
    p = oracle.rrs(X, Z, P, 600, 6, 0.7)["depth"]
    np.testing.assert_allclose(p, 1 / (1 + radii / q75), atol=tol * 2)
    a = oracle.rrs(X, Z, AP, 600, 6, 0.7)["depth"]
    np.testing.assert_allclose(a, 1 / (1 + radii / q75), atol=tol * 2)
    h = oracle.rrs(X, Z, H, 600, 6, 0.7)["depth"]
    np.testing.assert_allclose(h, 1 - norm.cdf(radii), atol=tol)


def test_rrs_one_round_is_simple_random_search():
    # Alg. S2 (simple random search): with r = 1 the search is the minimum of the univariate depth over k
    # directions drawn uniformly on the sphere, the lowest index winning ties.  The univariate depths here are
    # written out with numpy (median, unscaled MAD, halfspace counts), independently of the oracle's own.
    X, Z = workloads.gaussian_cloud(16, 301, 4, 5)
    k, seed = 64, 11
    for kind in (H, P):
        out = oracle.rrs(X, Z, kind, k, 1, 0.5, seed)
        for q in range(Z.shape[0]):
            U = oracle.directions(seed, q, 0, k, X.shape[1], 0.5).astype(np.float64)
            y = X @ U.T                                  # n x k projections
            yz = U @ Z[q]
            if kind == H:
                le = np.sum(y <= yz, axis=0)
                ge = np.sum(y >= yz, axis=0)
                c = np.minimum(le, ge)
                assert out["count"][q] == min(c.min(), X.shape[0])
                want_best = int(np.argmin(c)) if c.min() < X.shape[0] else -1
                assert out["best"][q] == want_best
            else:
                med = np.median(y, axis=0)
                mad = np.median(np.abs(y - med), axis=0)
                dj = 1.0 / (1.0 + np.abs(yz - med) / mad)
                np.testing.assert_allclose(out["depth"][q], min(dj.min(), 1.0), rtol=1e-12)
                assert out["best"][q] == int(np.argmin(dj))


def test_rrs_follow_mode_replays_own_choices():
    X, Z = workloads.gaussian_cloud(14, 400, 4, 6, dtype=np.float32)
    own = oracle.rrs(X, Z, P, 120, 6, 0.7, 3, rounds=True)
    # rebuild the update decisions from the per-round minima
    follow = np.full((Z.shape[0], 6), -1, np.int32)
    for q in range(Z.shape[0]):
        dmin = 1.0
        for l in range(6):
            if own["round_min"][q, l] < dmin:
                dmin = own["round_min"][q, l]
                follow[q, l] = own["round_arg"][q, l]
    rep = oracle.rrs(X, Z, P, 120, 6, 0.7, 3, follow=follow)
    np.testing.assert_array_equal(rep["depth"], own["depth"])
    np.testing.assert_array_equal(rep["best"], own["best"])


def test_rrs_query_index_keys_the_stream():
    X, Z = workloads.gaussian_cloud(15, 300, 3, 8)
    full = oracle.rrs(X, Z, H, 100, 5, 0.5, 21)
    sub = oracle.rrs(X, Z[[5, 2]], H, 100, 5, 0.5, 21, qidx=np.array([5, 2]))
    np.testing.assert_array_equal(sub["count"], full["count"][[5, 2]])
    np.testing.assert_array_equal(sub["best"], full["best"][[5, 2]])


def test_rrs_rejects_bad_arguments():
    X = np.zeros((3, 2))
    with pytest.raises(ValueError):
        oracle.rrs(X, X, H, 5, 10, 0.5)       # k < r
    with pytest.raises(ValueError):
        oracle.rrs(X, X, H, 10, 2, 1.5)       # alpha > 1


def _replay_depths(kind, X, z, U):
    """Univariate depths of z along the rows of U, written out here (Sec. 2): exact halfspace counts from
    rational arithmetic, projection / asymmetric projection depths from numpy FP64 medians."""
    from fractions import Fraction
    if kind == H:
        Xf = [[Fraction(float(v)) for v in row] for row in X]
        zf = [Fraction(float(v)) for v in z]
        out = []
        for u in U:
            uf = [Fraction(float(v)) for v in u]
            t = [sum(a * (b - c) for a, b, c in zip(uf, row, zf)) for row in Xf]
            le = sum(1 for v in t if v <= 0)
            ge = sum(1 for v in t if v >= 0)
            out.append(min(le, ge))
        return np.array(out, np.int64)
    y = X.astype(np.float64) @ U.astype(np.float64).T
    yz = U.astype(np.float64) @ z.astype(np.float64)
    med = np.median(y, axis=0)
    out = []
    for j in range(U.shape[0]):
        if kind == P:
            spread = np.median(np.abs(y[:, j] - med[j]))
            num = abs(yz[j] - med[j])
        else:
            pos = y[:, j][y[:, j] > med[j]] - med[j]
            spread = np.median(pos) if pos.size else 0.0
            num = max(yz[j] - med[j], 0.0)
        out.append((1.0 if num == 0 else 0.0) if spread == 0 else 1.0 / (1.0 + num / spread))
    return np.array(out)


def _replay_rrs(kind, X, z, q, k, r, alpha, seed):
    """Alg. 1 / Alg. S3 across rounds, written out here: round l draws its m directions about the current
    pole, the round minimum is taken at its lowest index, and D_min, the best flat index l*m + j* and the
    pole change only when the round minimum is strictly below D_min.  Returns (D_min, best, ties) where
    ties counts later rounds whose minimum equalled the running D_min (a non-strict update would move the
    best index there)."""
    n, d = X.shape
    m = -(-k // r)
    pole = np.zeros(d, np.float32)
    pole[0] = 1.0
    run = n if kind == H else 1.0
    best, ties = -1, 0
    for l in range(r):
        U = oracle.directions(seed, q, l, m, d, alpha, pole)
        v = _replay_depths(kind, X, z, U)
        ja = int(np.argmin(v))
        if v[ja] < run:
            run, best, pole = v[ja], l * m + ja, U[ja].copy()
        elif v[ja] == run and best >= 0:
            ties += 1
    return run, best, ties


def test_rrs_cross_round_update_is_strict():
    # Small integer clouds: halfspace counts take few values, so later rounds often tie the running minimum;
    # the oracle must keep the earlier best index and pole then (a <= update would move both).
    rng = np.random.default_rng(31)
    X = rng.integers(-5, 6, size=(12, 2)).astype(np.float64)
    Z = np.vstack([X[3], X[7], rng.integers(-3, 4, size=(4, 2)).astype(np.float64)])
    k, r, alpha, seed = 40, 5, 0.6, 5
    out = oracle.rrs(X, Z, H, k, r, alpha, seed)
    ties = 0
    for q in range(Z.shape[0]):
        run, best, t = _replay_rrs(H, X, Z[q], q, k, r, alpha, seed)
        ties += t
        assert out["count"][q] == run and out["best"][q] == best, q
        assert out["depth"][q] == run / X.shape[0]
    assert ties >= 3, "the case should exercise ties with the running minimum"


@pytest.mark.parametrize("kind", [P, AP])
def test_rrs_multi_round_replay_projection_depths(kind):
    # r = 6 rounds with shrinking caps about the moving pole; depths and best flat indices from the replay
    X, Z = workloads.gaussian_cloud(33 + kind, 257, 3, 6)
    k, r, alpha, seed = 60, 6, 0.7, 8
    out = oracle.rrs(X, Z, kind, k, r, alpha, seed)
    for q in range(Z.shape[0]):
        run, best, _ = _replay_rrs(kind, X, Z[q], q, k, r, alpha, seed)
        np.testing.assert_allclose(out["depth"][q], run, rtol=1e-12)
        assert out["best"][q] == best, q
