"""Seeded synthetic inputs for the RRS depth workloads.

This module only draws data clouds, query points and run parameters. It holds
none of the depth arithmetic, so both the CPU oracle (``oracle/``) and the GPU
path (``paper_2506_08262_gb300``) may use it without sharing any of the method.

The paper evaluates only on synthetic data (Gaussian clouds with a Toeplitz
covariance, Sec. 5; Student-t clouds, Sec. 7).  The five workloads below follow
the same recipe family:

* ``c1``: halfspace depth in d=2; X = 1,000 points ~ N(0, I_2) and 100 queries
  ~ N(0, 1.5^2 I_2), FP64; k = 1,000 directions as r = 10 rounds of 100, the cap
  angle halved every round (alpha = 0.5), direction seed 0.
* ``c2``: projection and asymmetric projection depth in d=10; X = 10,000 points,
  95% N(0, I_10) and 5% N(6*1, I_10), shuffled, FP32; 1,000 queries uniform in
  [-4, 4]^10; k = 1,000 over r = 20 rounds, alpha = 0.7.
* ``c3``: halfspace depth in d=50; X = 100,000 points whose coordinates are
  i.i.d. Student-t(3), mapped by the square root of a random SPD covariance
  (eigenvalues log-uniform in [0.1, 10], Haar eigenvectors); 10,000 queries
  from the same law; k = 2,000 over r = 20 rounds; alpha = 0.9 (the value the
  paper settles on in Sec. 5.1).
* ``c4``: 256 independent datasets, n log-uniform in [500, 50,000], d uniform
  in {5..100}, each N(mu_k, Sigma_k) with mu_k ~ U[-5, 5]^d and Sigma_k as in c3;
  1..1,000 queries per dataset from the same law; the depth kind drawn
  uniformly; k = 1,000 over r = 10 rounds, alpha = 0.9.
* ``c5``: 64 resident datasets drawn as in c4; Poisson arrivals at 2,000
  requests/s, each a batch of 1..4,096 queries (log-uniform), kinds mixed
  50/30/20 halfspace/projection/asymmetric; k = 1,000 over r = 10 rounds.

Every generator takes an explicit ``numpy.random.Generator`` seed; the default
data seed of workload ``cN`` is N.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

HALFSPACE = 0
PROJECTION = 1
ASYM_PROJECTION = 2
KIND_NAMES = {HALFSPACE: "halfspace", PROJECTION: "projection", ASYM_PROJECTION: "asymmetric"}


@dataclasses.dataclass
class Problem:
    """One dataset with its query batch and RRS parameters."""

    X: np.ndarray          # (n, d), float32 or float64, C-contiguous
    Z: np.ndarray          # (nq, d), same dtype as X
    kind: int              # HALFSPACE / PROJECTION / ASYM_PROJECTION
    k: int                 # total directions
    r: int                 # refinement rounds
    alpha: float           # cap shrink factor
    seed: int = 0          # direction-stream seed

    @property
    def n(self) -> int:
        return int(self.X.shape[0])

    @property
    def d(self) -> int:
        return int(self.X.shape[1])

    @property
    def nq(self) -> int:
        return int(self.Z.shape[0])

    @property
    def m(self) -> int:
        return -(-self.k // self.r)


def random_spd_sqrt(rng: np.random.Generator, d: int, lo: float = 0.1, hi: float = 10.0) -> np.ndarray:
    """Square root of a random SPD matrix: Q diag(sqrt(lam)) Q^T.

    Q is Haar-distributed (QR of a Gaussian matrix with the sign of R's diagonal
    fixed) and lam is log-uniform in [lo, hi].
    """
    G = rng.standard_normal((d, d))
    Qm, R = np.linalg.qr(G)
    Qm = Qm * np.sign(np.diag(R))[None, :]
    lam = np.exp(rng.uniform(math.log(lo), math.log(hi), size=d))
    return (Qm * np.sqrt(lam)[None, :]) @ Qm.T


def c1(seed: int = 1, n: int = 1000, nq: int = 100) -> Problem:
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, 2))
    Z = 1.5 * rng.standard_normal((nq, 2))
    return Problem(np.ascontiguousarray(X), np.ascontiguousarray(Z), HALFSPACE, 1000, 10, 0.5, 0)


def c2(seed: int = 2, n: int = 10_000, nq: int = 1000, kind: int = PROJECTION) -> Problem:
    rng = np.random.default_rng(seed)
    d = 10
    n_out = n // 20
    X = np.concatenate([rng.standard_normal((n - n_out, d)),
                        6.0 + rng.standard_normal((n_out, d))])
    X = X[rng.permutation(n)]
    Z = rng.uniform(-4.0, 4.0, size=(nq, d))
    return Problem(np.ascontiguousarray(X, dtype=np.float32), np.ascontiguousarray(Z, dtype=np.float32),
                   kind, 1000, 20, 0.7, 0)


def c2_queries(rank: int, nq: int = 1000) -> np.ndarray:
    """The projection-depth workload's queries taken by rank `rank` of a multi-GPU run: rank 0 the
    workload's own, every other rank nq fresh draws from the same law U[-4,4]^10 seeded by (2, rank), so the
    ranks share the data cloud and no query repeats across ranks."""
    if rank == 0:
        return c2(nq=nq).Z
    rng = np.random.default_rng([2, rank])
    return np.ascontiguousarray(rng.uniform(-4.0, 4.0, size=(nq, 10)), dtype=np.float32)


def c3(seed: int = 3, n: int = 100_000, nq: int = 10_000, d: int = 50) -> Problem:
    rng = np.random.default_rng(seed)
    A = random_spd_sqrt(rng, d)
    X = rng.standard_t(3.0, size=(n, d)) @ A.T
    Z = rng.standard_t(3.0, size=(nq, d)) @ A.T
    return Problem(np.ascontiguousarray(X, dtype=np.float32), np.ascontiguousarray(Z, dtype=np.float32),
                   HALFSPACE, 2000, 20, 0.9, 0)


def _gaussian_dataset(rng: np.random.Generator, n: int, d: int, nq: int):
    mu = rng.uniform(-5.0, 5.0, size=d)
    A = random_spd_sqrt(rng, d)
    X = mu + rng.standard_normal((n, d)) @ A.T
    Z = mu + rng.standard_normal((nq, d)) @ A.T
    return (np.ascontiguousarray(X, dtype=np.float32), np.ascontiguousarray(Z, dtype=np.float32))


def c4(seed: int = 4, n_datasets: int = 256, n_lo: int = 500, n_hi: int = 50_000,
       q_hi: int = 1000, scale: float = 1.0) -> List[Problem]:
    """Batched workload; ``scale`` < 1 shrinks n and the query counts for tests."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_datasets):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        n = max(1, int(n * scale))
        d = int(rng.integers(5, 101))
        nq = max(1, int(int(rng.integers(1, q_hi + 1)) * scale))
        kind = int(rng.integers(0, 3))
        X, Z = _gaussian_dataset(rng, n, d, nq)
        out.append(Problem(X, Z, kind, 1000, 10, 0.9, 0))
    return out


@dataclasses.dataclass
class Request:
    t_arrival: float       # seconds from the start of the window
    dataset: int           # index into the resident datasets
    Z: np.ndarray          # (nq, d) float32
    kind: int


def c5(seed: int = 5, n_datasets: int = 64, rate: float = 2000.0, window_s: float = 1.0,
       q_hi: int = 4096, n_hi: int = 50_000, scale: float = 1.0):
    """Serving workload: resident datasets plus a Poisson request stream."""
    rng = np.random.default_rng(seed)
    datasets = []
    for _ in range(n_datasets):
        n = int(round(math.exp(rng.uniform(math.log(500), math.log(n_hi)))))
        n = max(1, int(n * scale))
        d = int(rng.integers(5, 101))
        mu = rng.uniform(-5.0, 5.0, size=d)
        A = random_spd_sqrt(rng, d)
        X = mu + rng.standard_normal((n, d)) @ A.T
        datasets.append((np.ascontiguousarray(X, dtype=np.float32), mu, A))
    reqs = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= window_s:
            break
        ds = int(rng.integers(0, n_datasets))
        nq = int(round(math.exp(rng.uniform(0.0, math.log(q_hi)))))
        nq = max(1, int(nq * scale))
        kind = int(rng.choice(3, p=[0.5, 0.3, 0.2]))
        _, mu, A = datasets[ds]
        Z = mu + rng.standard_normal((nq, A.shape[0])) @ A.T
        reqs.append(Request(t, ds, np.ascontiguousarray(Z, dtype=np.float32), kind))
    return [X for X, _, _ in datasets], reqs


def gaussian_cloud(seed: int, n: int, d: int, nq: int, dtype=np.float64, zscale: float = 1.0):
    """Plain N(0, I_d) cloud and N(0, zscale^2 I_d) queries (small parity cases)."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d))
    Z = zscale * rng.standard_normal((nq, d))
    return np.ascontiguousarray(X, dtype=dtype), np.ascontiguousarray(Z, dtype=dtype)


def toeplitz_scatter(d: int) -> np.ndarray:
    """The paper's Toeplitz matrix sigma_ij = 2^{-|i-j|} (Sec. 5)."""
    idx = np.arange(d)
    return 2.0 ** (-np.abs(idx[:, None] - idx[None, :]))


def ranking_cloud(seed: int, n: int, d: int, nu: float, npts: int, dtype=np.float32):
    """The center-outward ranking data of Sec. 6: n points of N(0, S) (nu = inf) or of the multivariate
    Student-t with nu degrees of freedom and scatter S (a N(0, S) draw divided by sqrt(w / nu), w ~ chi2_nu),
    S = toeplitz_scatter(d), and npts of them chosen at random as query points.  Returns (X, Z, S)."""
    rng = np.random.default_rng(seed)
    S = toeplitz_scatter(d)
    L = np.linalg.cholesky(S)
    X = rng.standard_normal((n, d)) @ L.T
    if np.isfinite(nu):
        X = X / np.sqrt(rng.chisquare(nu, size=n) / nu)[:, None]
    idx = rng.choice(n, size=npts, replace=False)
    X = np.ascontiguousarray(X, dtype=dtype)
    return X, np.ascontiguousarray(X[idx]), S


def toeplitz_gaussian(seed: int, n: int, d: int, nq: int, dtype=np.float32):
    """N(0, Sigma) with sigma_ij = 2^{-|i-j|} (the paper's Sec. 5 generator)."""
    rng = np.random.default_rng(seed)
    idx = np.arange(d)
    S = 2.0 ** (-np.abs(idx[:, None] - idx[None, :]))
    L = np.linalg.cholesky(S)
    X = rng.standard_normal((n, d)) @ L.T
    Z = rng.standard_normal((nq, d)) @ L.T
    return np.ascontiguousarray(X, dtype=dtype), np.ascontiguousarray(Z, dtype=dtype)
