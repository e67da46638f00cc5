"""Seeded synthetic inputs shaped like the paper's workloads (Sec. VII).

This module draws random numbers only: locations on a jittered grid, standard
normal vectors e, hold-out index sets and per-region parameter draws.  It holds
none of the method's arithmetic (no covariance, no factorisation), so both the
CUDA path and the CPU oracle may import it.

Sec. VII defines the synthetic locations as n^{-1/2}(r - 0.5 + X_rl, l - 0.5 + Y_rl)
with X, Y ~ U(-0.4, 0.4) and r, l in {1..sqrt(n)}; the printed formula multiplies
by n^{1/2}, which would put the points in [0, sqrt(n)]^2 and contradict the
range values 0.03/0.1/0.3 of Sec. IV, so the points are divided by the grid side
and land in [0, 1]^2.
"""
from __future__ import annotations

import numpy as np

SEED = 20241  # base seed of every synthetic workload

# independent streams derived from the base seed
STREAM_LOCATIONS = 0
STREAM_NOISE = 1
STREAM_HOLDOUT = 2
STREAM_REGIONS = 3
STREAM_NEW_POINTS = 4


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([seed, stream])


def jittered_grid(side: int, seed: int = SEED, n: int | None = None):
    """Locations of a side x side jittered grid in [0,1]^2 (Sec. VII).

    Returns (x, y) as float64 arrays of length side*side, or of length ``n``
    when ``n`` is given (a seeded random subset of the grid, used when n is not
    a perfect square).
    """
    rng = _rng(seed, STREAM_LOCATIONS)
    r, l = np.meshgrid(np.arange(1, side + 1), np.arange(1, side + 1), indexing="ij")
    X = rng.uniform(-0.4, 0.4, size=(side, side))
    Y = rng.uniform(-0.4, 0.4, size=(side, side))
    x = ((r - 0.5 + X) / side).ravel()
    y = ((l - 0.5 + Y) / side).ravel()
    if n is not None and n < side * side:
        keep = np.sort(rng.choice(side * side, size=n, replace=False))
        x, y = x[keep], y[keep]
    return np.ascontiguousarray(x), np.ascontiguousarray(y)


def locations(n: int, seed: int = SEED):
    """n jittered-grid locations; side = ceil(sqrt(n)), subset when not square."""
    side = int(np.ceil(np.sqrt(n) - 1e-9))
    return jittered_grid(side, seed, n if side * side != n else None)


def uniform_points(m: int, seed: int = SEED):
    """m prediction locations drawn uniformly on [0,1]^2 (not on the grid)."""
    rng = _rng(seed, STREAM_NEW_POINTS)
    p = rng.uniform(0.0, 1.0, size=(2, m))
    return np.ascontiguousarray(p[0]), np.ascontiguousarray(p[1])


def standard_normal(n: int, seed: int = SEED, stream: int = STREAM_NOISE) -> np.ndarray:
    """e ~ N(0, I_n) in float64, the white noise behind z = L e (Sec. VIII-D)."""
    return _rng(seed, stream).standard_normal(n)


def holdout(n: int, m: int, seed: int = SEED):
    """Split {0..n-1} into (observed, held_out) index arrays, |held_out| = m."""
    rng = _rng(seed, STREAM_HOLDOUT)
    held = np.sort(rng.choice(n, size=m, replace=False))
    mask = np.ones(n, dtype=bool)
    mask[held] = False
    return np.nonzero(mask)[0], held


def region_draws(R: int = 512, seed: int = SEED, n_lo: int = 500, n_hi: int = 8000):
    """Per-region sizes and parameters of the batched-regions workload.

    n_r ~ U{n_lo..n_hi}, sigma^2 ~ U[0.5, 2], beta ~ U[0.03, 0.3], nu uniform on
    {0.5, 1.0, 1.5}.
    """
    rng = _rng(seed, STREAM_REGIONS)
    n = rng.integers(n_lo, n_hi + 1, size=R)
    sigma2 = rng.uniform(0.5, 2.0, size=R)
    beta = rng.uniform(0.03, 0.3, size=R)
    nu = rng.choice(np.array([0.5, 1.0, 1.5]), size=R)
    return n, np.stack([sigma2, beta, nu], axis=1)
