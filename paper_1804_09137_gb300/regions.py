"""Batched independent regions and a measured tile-size autotuner.

Many unrelated likelihood problems (for instance the regions of a large field,
each with its own exact MLE, Sec. VII-VIII) are evaluated by
``tlr.loglik_grad_batched``.  The tile size nb trades arithmetic intensity
against parallelism (Sec. V); ``autotune_nb`` picks it per size class by
timing one synthetic problem of the class at each candidate (a single tile,
nb >= n, is the dense path) together with the rank cap.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import inputs
from . import tlr as T

DEFAULT_CANDIDATES = (0, 384, 512, 768, 1024)  # 0: one tile covering the region (dense)


def size_class(n: int, edges=(2000, 4000)) -> int:
    return int(np.searchsorted(np.asarray(edges), n, side="right"))


def _time_one(n, nb, eps, theta, dev, reps=2, rank_cap=None):
    x, y = inputs.locations(n, seed=1234)
    t = lambda a: torch.tensor(a, dtype=torch.float64, device=dev)
    nb_eff = n if nb <= 0 or nb >= n else nb
    cap = max(nb_eff // 2, 16) if rank_cap is None else rank_cap
    h = T.Handle(t(x), t(y), nb=nb_eff, eps=eps, rank_cap=cap)
    z = t(inputs.standard_normal(n, seed=1234))
    best = float("inf")
    try:
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h.factor(theta)
            h.loglik_grad(z)
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t0)
        h.check()
    except T.TlrError:  # e.g. the rank cap is exceeded: not a valid candidate
        best = float("inf")
    h.close()
    return best


def autotune_nb(sizes, eps: float, theta=(1.0, 0.1, 1.0), candidates=DEFAULT_CANDIDATES, edges=(2000, 4000),
                dev=None, cap_fracs=(0.25, 0.5)):
    """{size class: (nb, rank_cap, seconds, {(nb, rank_cap): seconds})} measured on the median-size region of
    each class: every tile size with every rank cap nb * f, f in cap_fracs (a single tile, nb = 0, has
    none); a candidate that fails (rank cap exceeded) is not chosen."""
    dev = dev or torch.device("cuda")
    sizes = np.asarray(sizes)
    classes = np.array([size_class(int(v), edges) for v in sizes])
    out = {}
    for c in np.unique(classes):
        n_med = int(np.median(sizes[classes == c]))
        timings = {}
        for nb in candidates:
            if 0 < nb and nb * 2 > n_med:  # fewer than two tiles: same as the dense single tile
                continue
            caps = [0] if nb <= 0 else sorted({max(int(nb * f), 16) for f in cap_fracs})
            for cap in caps:
                timings[(nb, cap)] = _time_one(n_med, nb, eps, theta, dev, rank_cap=cap if cap else None)
        best = min(timings, key=timings.get)
        out[int(c)] = (int(best[0]), int(best[1]), float(timings[best]),
                       {k: float(v) for k, v in timings.items()})
    return out


def make_opts(n, nb_choice, eps, edges=(2000, 4000)):
    """TlrOpts per region from the autotuned choice of its size class."""
    nb, cap, _, _ = nb_choice[size_class(int(n), edges)]
    if nb <= 0 or nb >= n:
        return T.TlrOpts(int(n), float(eps), 0, 0, 1, 0, 0.0)
    return T.TlrOpts(int(nb), float(eps), int(cap) if cap > 0 else max(nb // 2, 16), 0, 1, 0, 0.0)


def region_problems(R=512, seed=inputs.SEED, n_lo=500, n_hi=8000):
    """Seeded regions: sizes, thetas and jittered-grid points on each region's unit square."""
    sizes, thetas = inputs.region_draws(R, seed, n_lo, n_hi)
    pts = [inputs.locations(int(n), seed=seed + 1 + r) for r, n in enumerate(sizes)]
    return sizes, thetas, pts
