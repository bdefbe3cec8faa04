"""The synthetic input recipes: each generator draws what its docstring and the
benchmark's workload strings state (shapes, dtypes, mixture proportions, query
ranges, spectra, size ranges), and the same seed gives the same arrays."""
import math

import numpy as np

import workloads


def test_c1_shapes_and_query_spread():
    P = workloads.c1()
    assert P.X.shape == (1000, 2) and P.Z.shape == (100, 2) and P.X.dtype == np.float64
    assert (P.kind, P.k, P.r, P.alpha) == (workloads.HALFSPACE, 1000, 10, 0.5)
    # queries ~ N(0, 1.5^2 I): sample std within a few standard errors
    assert abs(P.Z.std() - 1.5) < 0.15 and abs(P.X.std() - 1.0) < 0.05


def test_c2_mixture_and_query_box():
    P = workloads.c2()
    assert P.X.shape == (10_000, 10) and P.Z.shape == (1000, 10) and P.X.dtype == np.float32
    assert (P.k, P.r, P.alpha, P.m) == (1000, 20, 0.7, 50)
    # 5% of the rows come from N(6 * 1, I): their coordinate mean is near 6, the rest near 0
    far = P.X.mean(axis=1) > 3.0
    assert far.sum() == 500
    assert abs(P.X[far].mean() - 6.0) < 0.1 and abs(P.X[~far].mean()) < 0.05
    assert not far[:500].all()                     # shuffled, not stacked
    assert P.Z.min() >= -4.0 and P.Z.max() <= 4.0


def test_spd_square_root_spectrum():
    rng = np.random.default_rng(0)
    A = workloads.random_spd_sqrt(rng, 50)
    np.testing.assert_allclose(A, A.T, atol=1e-12)
    lam = np.linalg.eigvalsh(A @ A)
    assert lam.min() >= 0.1 * (1 - 1e-9) and lam.max() <= 10.0 * (1 + 1e-9)


def test_c3_student_t_law_small():
    P = workloads.c3(n=20_000, nq=100)
    assert P.X.shape == (20_000, 50) and P.Z.shape == (100, 50) and P.X.dtype == np.float32
    assert (P.kind, P.k, P.r, P.alpha) == (workloads.HALFSPACE, 2000, 20, 0.9)
    # t(3) has variance 3, so the covariance of X is 3 A A' with eigenvalues in [0.3, 30]
    lam = np.linalg.eigvalsh(np.cov(P.X.astype(np.float64).T))
    assert lam.min() > 0.2 and lam.max() < 45.0


def test_c4_sizes_kinds_and_scale():
    probs = workloads.c4(n_datasets=64, scale=0.05)
    assert len(probs) == 64
    for P in probs:
        assert 1 <= P.n <= 2500 and 5 <= P.d <= 100 and 1 <= P.nq <= 50
        assert P.kind in (0, 1, 2) and (P.k, P.r, P.alpha) == (1000, 10, 0.9)
    assert {P.kind for P in probs} == {0, 1, 2}
    full = workloads.c4(n_datasets=8, scale=1.0)
    assert all(500 <= P.n <= 50_000 for P in full)


def test_c5_arrivals_and_kind_mix():
    datasets, reqs = workloads.c5(n_datasets=4, rate=2000.0, window_s=1.0, scale=0.01)
    assert len(datasets) == 4
    # Poisson arrivals at 2,000/s over 1 s: about 2,000 requests, increasing times inside the window
    assert abs(len(reqs) - 2000) < 5 * math.sqrt(2000)
    t = np.array([r.t_arrival for r in reqs])
    assert np.all(np.diff(t) > 0) and t[-1] < 1.0
    kinds = np.bincount([r.kind for r in reqs], minlength=3) / len(reqs)
    np.testing.assert_allclose(kinds, [0.5, 0.3, 0.2], atol=0.05)
    assert all(r.Z.shape[1] == datasets[r.dataset].shape[1] for r in reqs)


def test_ranking_cloud_scatter_and_queries_from_the_cloud():
    X, Z, S = workloads.ranking_cloud(1, 40_000, 5, np.inf, 30)
    np.testing.assert_allclose(S[0], [1.0, 0.5, 0.25, 0.125, 0.0625])
    np.testing.assert_allclose(np.cov(X.astype(np.float64).T), S, atol=0.03)
    rows = {r.tobytes() for r in X}
    assert all(z.tobytes() in rows for z in Z)
    Xt, _, _ = workloads.ranking_cloud(2, 40_000, 5, 5.0, 3)
    # multivariate t with nu = 5 and scatter S has covariance nu / (nu - 2) S
    np.testing.assert_allclose(np.cov(Xt.astype(np.float64).T)[0, 0], 5.0 / 3.0, rtol=0.1)


def test_generators_are_seeded():
    a, b = workloads.c2(), workloads.c2()
    np.testing.assert_array_equal(a.X, b.X)
    np.testing.assert_array_equal(a.Z, b.Z)
    assert not np.array_equal(workloads.c2(seed=3).X, a.X)
