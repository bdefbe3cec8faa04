"""Exact references used to pin the oracle (test infrastructure only).

* ``halfspace_depth_2d``: the exact (infimum over all directions) Tukey depth
  of a point in the plane, by brute force in O(n^2) per query.  Between two
  consecutive critical directions (u orthogonal to some x_i - z) the two closed
  halfspace counts of Sec. 2 are constant, and at a critical direction they can
  only be larger (a boundary point counts on both sides), so the infimum is
  reached inside an open arc: it suffices to count at the midpoint of every
  arc between sorted critical angles.  Signs at the midpoints are decided with
  an FP64 forward error bound and, where that is inconclusive, with exact
  rational arithmetic.
* ``sign_fraction`` / ``univariate_fraction``: the univariate depths of Sec. 2
  in exact rational arithmetic for tiny inputs (Python ``fractions``).
"""
from __future__ import annotations

import math
from fractions import Fraction
from typing import Sequence

import numpy as np


def sign_fraction(u: Sequence[float], x: Sequence[float], z: Sequence[float]) -> int:
    """Exact sign of u^T (x - z) for binary floating-point entries."""
    t = Fraction(0)
    for ul, xl, zl in zip(u, x, z):
        t += Fraction(float(ul)) * (Fraction(float(xl)) - Fraction(float(zl)))
    return (t > 0) - (t < 0)


def _median_fraction(v):
    v = sorted(v)
    L = len(v)
    if L % 2:
        return v[(L - 1) // 2]
    return (v[L // 2 - 1] + v[L // 2]) / 2


def univariate_fraction(kind: int, X, z, u):
    """Depth of z along u in exact arithmetic (kind 0/1/2 = H/P/AP).

    Returns a Fraction for kinds 0 and the exact rational value of the
    projection depth formula for kinds 1 and 2 (the readings of the oracle:
    unscaled MAD, strict positive deviations, zero-MAD limits)."""
    uf = [Fraction(float(a)) for a in u]
    y = [sum(a * Fraction(float(b)) for a, b in zip(uf, row)) for row in X]
    yz = sum(a * Fraction(float(b)) for a, b in zip(uf, z))
    n = len(y)
    if kind == 0:
        le = sum(1 for v in y if v <= yz)
        ge = sum(1 for v in y if v >= yz)
        return Fraction(min(le, ge), n)
    med = _median_fraction(y)
    if kind == 1:
        mad = _median_fraction([abs(v - med) for v in y])
        num = abs(yz - med)
    else:
        pos = [v - med for v in y if v > med]
        mad = _median_fraction(pos) if pos else Fraction(0)
        num = max(yz - med, Fraction(0))
    if mad == 0:
        return Fraction(1) if num == 0 else Fraction(0)
    return 1 / (1 + num / mad)


def _sign_at(c: float, s: float, X: np.ndarray, z: np.ndarray, dx: np.ndarray,
             dy: np.ndarray) -> np.ndarray:
    """Exact signs of (c, s)^T (x_i - z); dx, dy are the FP64-rounded differences."""
    t = c * dx + s * dy
    bound = 8.0 * 2.0 ** -53 * (abs(c) * np.abs(dx) + abs(s) * np.abs(dy))
    sg = np.where(t > bound, 1, np.where(t < -bound, -1, 2))
    for i in np.nonzero(sg == 2)[0]:
        sg[i] = sign_fraction((c, s), X[i], z)
    return sg


def halfspace_count_2d(X: np.ndarray, z: np.ndarray) -> int:
    """min over all directions of min(#{u'x <= u'z}, #{u'x >= u'z}), d = 2."""
    X = np.asarray(X, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    n = X.shape[0]
    dx = X[:, 0] - z[0]
    dy = X[:, 1] - z[1]
    at_z = np.array([X[i, 0] == z[0] and X[i, 1] == z[1] for i in range(n)])
    if int(at_z.sum()) == n:
        return n
    phi = np.arctan2(dy[~at_z], dx[~at_z])
    crit = np.concatenate([phi + math.pi / 2, phi - math.pi / 2]) % (2 * math.pi)
    crit = np.sort(crit)
    gaps = np.diff(np.concatenate([crit, [crit[0] + 2 * math.pi]]))
    tiny = gaps[(gaps > 0) & (gaps < 1e-9)]
    if tiny.size:
        raise ValueError("critical angles closer than 1e-9 rad: input too degenerate")
    best = n
    for a, g in zip(crit, gaps):
        if g == 0.0:
            continue  # coincident critical angles: the arc has no interior
        mid = a + g / 2
        c, s = math.cos(mid), math.sin(mid)
        sg = _sign_at(c, s, X, z, dx, dy)
        lt = int((sg < 0).sum())
        gt = int((sg > 0).sum())
        best = min(best, n - gt, n - lt)
    return best


def halfspace_depth_2d(X: np.ndarray, Z: np.ndarray) -> np.ndarray:
    """Exact 2-D halfspace counts (integers) for every row of Z."""
    Z = np.asarray(Z, dtype=np.float64).reshape(-1, 2)
    return np.array([halfspace_count_2d(X, z) for z in Z], dtype=np.int64)
