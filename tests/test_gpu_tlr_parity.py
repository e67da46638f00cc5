"""GPU parity at the working threshold: the paths the n = 90,000 benchmark runs, against the oracle.

* The Morton permutation of the library (tlr_get_perm) equals oracle.tlr.morton_permutation bit for bit
  (index work), including ties and non-square point counts.
* l and dl/dtheta at eps = 1e-7 with low-rank tiles in L and in L^{-1} (tile size 900 as in the benchmark,
  and 256), compared with the exact dense float64 oracle values of tests/golden/tlr_parity.json, on points
  at the benchmark's density so that the tiles have its spatial extent and ranks.

Tolerances.  l: the metric's relative 1e-6 at eps = 1e-7, or, where the tile low-rank method itself does
not reach it on these points, the error of the CPU TLR reference (oracle.tlr, SVD truncation at the same eps)
against the exact value; each of the terms log|Sigma| / 2 and z^T Sigma^{-1} z / 2 within that budget on its
own.  At eps = 1e-9 the same with 1e-8 (first order: a hundred times smaller).  dl/dtheta, two criteria:
  * the acceptance criterion on the estimate: a gradient error dg moves the maximum-likelihood estimate by
    -H^{-1} dg (H the Hessian of l, from the oracle); that shift must stay within 1% of theta per component;
  * first order in the thresholds: the gradient's error comes from the truncations at eps (Cholesky,
    Sec. V) and at inv_scale * eps * zeta^(1/2) (L^{-1}), both linear in eps, so at eps = 1e-9 the error
    must be at least ten times smaller than at 1e-7 (one hundred times to first order), or below
    1e-8 |grad|.
Worst-case first-order bounds built from norms of Sigma^{-1} exceed the gradient itself at these sizes, so
they pin nothing; the measured errors are reported with the benchmark.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dense as DN
from oracle import tlr as TL
from paper_1804_09137_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "tlr_parity.json")


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g

    g.build()
    from paper_1804_09137_gb300 import tlr

    return tlr


def dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda")


def _perm(T, x, y):
    h = T.Handle(dev(x), dev(y), nb=64, eps=1e-9)
    p = h.get_perm().cpu().numpy().astype(np.int64)
    h.close()
    return p


@pytest.mark.parametrize("side,n", [(30, None), (37, 1200), (64, 4000)])
def test_morton_permutation_is_bit_exact(T, side, n):
    x, y = inputs.jittered_grid(side, n=n)
    np.testing.assert_array_equal(_perm(T, x, y), TL.morton_permutation(x, y))


def test_morton_permutation_ties_and_offsets(T):
    # duplicated points and points that share a quantisation cell keep their input order; a bounding
    # box that is not a square and does not start at the origin
    x, y = inputs.jittered_grid(20)
    x = 3.0 + 2.0 * x
    y = -1.0 + 0.5 * y
    x = np.concatenate([x, x[:17], x[5:9] + 1e-12])
    y = np.concatenate([y, y[:17], y[5:9]])
    p = _perm(T, x, y)
    np.testing.assert_array_equal(p, TL.morton_permutation(x, y))
    first = {int(v): i for i, v in enumerate(p)}
    assert all(first[i] < first[len(x) - 21 + i] for i in range(17))


def _golden(name):
    with open(GOLDEN) as fh:
        return json.load(fh)[name]


def _run(T, g, eps, rank_cap, dense_rank, precision=0):
    x, y = inputs.jittered_grid(g["side"], n=g["subset"])
    x, y = x * g["scale"], y * g["scale"]
    theta = tuple(g["theta"])
    z = DN.sample(x, y, theta, inputs.standard_normal(len(x)))
    nb = g["nb"]
    h = T.Handle(dev(x), dev(y), nb=nb, eps=eps, rank_cap=rank_cap, dense_rank=dense_rank, precision=precision)
    assert h.nt >= 5 and len(x) % nb != 0  # several tiles, the last one ragged
    h.factor(theta)
    zt = dev(z)
    out = h.loglik(zt).cpu().numpy()
    ll, grad = h.loglik_grad(zt)
    h.check()
    info = {"tiles": h.tile_counts(), "inverse": h.inverse_stats(), "nt": h.nt}
    h.close()
    return out, float(ll.item()), grad.cpu().numpy(), info


@pytest.mark.parametrize("name,rank_cap,dense_rank", [("nb900", 256, 0), ("nb256", 128, 96)])
def test_working_eps_loglik_and_gradient_match_oracle(T, name, rank_cap, dense_rank):
    g = _golden(name)
    gref = np.array(g["grad"])
    out, ll, grad, info = _run(T, g, 1e-7, rank_cap, dense_rank)
    # most off-diagonal tiles of L and of L^{-1} are low rank: the truncated paths ran
    ntiles = info["nt"] * (info["nt"] - 1) // 2
    assert info["tiles"]["lowrank"] > ntiles // 2, info
    assert ntiles - info["inverse"]["dense"] > ntiles // 2, info
    assert info["inverse"]["kmax"] > 0
    assert abs(ll - out[0]) <= 1e-12 * abs(out[0])
    tol = max(1e-6 * abs(g["loglik"]), abs(g["tlr_ref"]["1e-07"][0] - g["loglik"]))
    assert abs(ll - g["loglik"]) <= tol, (ll, g["loglik"], tol)
    # l = c - log|Sigma| / 2 - q / 2: each term within the budget for l on its own (no cancellation)
    assert 0.5 * abs(out[1] - g["logdet"]) <= tol
    assert 0.5 * abs(out[2] - g["quad"]) <= tol
    err7 = np.linalg.norm(grad - gref)
    shift = -np.linalg.solve(np.array(g["hessian"]), grad - gref)
    assert np.all(np.abs(shift) <= 0.01 * np.abs(np.array(g["theta"]))), (grad, gref, shift)
    # first order in eps: a hundred times smaller thresholds, at least ten times smaller error
    _, ll9, grad9, _ = _run(T, g, 1e-9, rank_cap, dense_rank)
    err9 = np.linalg.norm(grad9 - gref)
    assert err9 <= max(0.1 * err7, 1e-8 * np.linalg.norm(gref)), (err9, err7)
    tol9 = max(1e-8 * abs(g["loglik"]), abs(g["tlr_ref"]["1e-09"][0] - g["loglik"]))
    assert abs(ll9 - g["loglik"]) <= tol9, (ll9, g["loglik"], tol9)


@pytest.mark.parametrize("precision", [5, 1])
def test_other_precisions_stay_within_the_working_eps_budget(T, precision):
    """precision 5 (mixed: 5 bf16 slices, tensor cores also in the Cholesky) and 1 (double-float only) at
    eps = 1e-7 on the nb = 900 case: l within the same budget as the default, the gradient's MLE shift
    within 1 % of theta."""
    g = _golden("nb900")
    gref = np.array(g["grad"])
    out, ll, grad, _ = _run(T, g, 1e-7, 256, 0, precision)
    tol = max(1e-6 * abs(g["loglik"]), abs(g["tlr_ref"]["1e-07"][0] - g["loglik"]))
    assert abs(ll - g["loglik"]) <= tol, (ll, g["loglik"], tol)
    shift = -np.linalg.solve(np.array(g["hessian"]), grad - gref)
    assert np.all(np.abs(shift) <= 0.01 * np.abs(np.array(g["theta"]))), (grad, gref, shift)


def test_sigma2_derivative_matches_finite_differences_of_gpu_loglik(T):
    """dl/dsigma2 at eps = 1e-7 against central differences of the library's own l in sigma2 (n = 1,600).
    Sigma = sigma2 R: every tile scales with sigma2, so the ranks do not change over the step and the
    TLR l is smooth in sigma2 there."""
    theta = np.array([1.0, 0.3, 1.0])
    x, y = inputs.jittered_grid(40)
    z = DN.sample(x, y, tuple(theta), inputs.standard_normal(len(x)))
    h = T.Handle(dev(x), dev(y), nb=200, eps=1e-7, rank_cap=100)
    zt = dev(z)
    h.factor(theta)
    _, g = h.loglik_grad(zt)
    h.check()
    g0 = float(g[0].item())
    hs = 1e-4
    vals = []
    for sgn in (1, -1):
        th = theta.copy()
        th[0] += sgn * hs
        h.factor(th)
        vals.append(float(h.loglik(zt)[0].item()))
        h.check()
    fd = (vals[0] - vals[1]) / (2 * hs)
    # central difference truncation ~ h^2 |l'''| / 6 with l''' = O(n / sigma2^3); rounding ~ 1e-15 |l| / h
    assert abs(g0 - fd) <= 1e-5 * max(abs(fd), 1.0), (g0, fd)
    h.close()
