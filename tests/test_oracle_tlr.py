"""Pins of oracle/tlr.py (Sec. V tile low-rank format and TLR Cholesky)."""
import numpy as np
import pytest
import scipy.linalg as sl

from oracle import dense as DN
from oracle import tlr as TL
from paper_1804_09137_gb300 import inputs

TH = (1.0, 0.1, 0.5)


def _problem(side, theta=TH, n=None):
    x, y = inputs.jittered_grid(side, n=n)
    z = DN.sample(x, y, theta, inputs.standard_normal(len(x)))
    return x, y, z


def test_morton_is_permutation_and_quadrants():
    # on a 4x4 regular grid the first 4 points of the Z-curve are one 2x2 quadrant
    g = (np.arange(4) + 0.5) / 4
    X, Y = np.meshgrid(g, g, indexing="ij")
    x, y = X.ravel(), Y.ravel()
    p = TL.morton_permutation(x, y)
    assert sorted(p) == list(range(16))
    for q in range(4):
        blk = p[4 * q:4 * q + 4]
        assert np.ptp(x[blk]) < 0.3 and np.ptp(y[blk]) < 0.3


def test_compress_threshold_rule():
    x, y, _ = _problem(16)
    p = TL.morton_permutation(x, y)
    S = DN.covariance(x[p], y[p], (1.0, 0.3, 1.0))
    eps = 1e-6
    T = TL.compress(S, 64, eps)
    for (i, j), U in T.U.items():
        A = S[T.rows(i), T.rows(j)]
        E = A - U @ T.V[i, j].T
        assert np.linalg.norm(E, 2) <= eps * (1 + 1e-9)
        k = U.shape[1]
        if k > 0:  # the last kept direction was needed: its singular value exceeds eps
            assert np.linalg.svd(U @ T.V[i, j].T, compute_uv=False)[k - 1] > eps


@pytest.mark.parametrize("theta", [(1.0, 0.1, 0.5), (1.0, 0.3, 1.0)])
def test_eps_zero_equals_dense(theta):
    x, y, z = _problem(18, theta, n=300)
    ll_d = DN.loglik(x, y, z, theta)
    ll_t = TL.loglik(x, y, z, theta, nb=64, eps=0.0)
    assert abs(ll_t[0] - ll_d[0]) <= 1e-10 * abs(ll_d[0])
    assert abs(ll_t[1] - ll_d[1]) <= 1e-10 * abs(ll_d[1])


def test_single_tile_is_dense():
    x, y, z = _problem(10)
    ll_d = DN.loglik(x, y, z, TH)[0]
    ll_t = TL.loglik(x, y, z, TH, nb=200, eps=1e-3)[0]
    assert abs(ll_t - ll_d) <= 1e-13 * abs(ll_d)


def test_factor_reconstructs_sigma():
    x, y, z = _problem(16)
    T, p = TL.factor(x, y, TH, nb=48, eps=1e-10)
    n, nb = len(x), 48
    L = np.zeros((n, n))
    for i in range(T.nt):
        L[T.rows(i), T.rows(i)] = T.D[i]
        for j in range(i):
            L[T.rows(i), T.rows(j)] = T.U[i, j] @ T.V[i, j].T
    S = DN.covariance(x[p], y[p], TH)
    assert np.linalg.norm(L @ L.T - S, 2) <= 1e-7
    # tile solves equal dense triangular solves on the assembled factor
    w = TL.forward_solve(T, z[p])
    np.testing.assert_allclose(w, sl.solve_triangular(L, z[p], lower=True), rtol=1e-10, atol=1e-10)
    v = TL.backward_solve(T, w)
    np.testing.assert_allclose(v, sl.solve_triangular(L, w, lower=True, trans="T"), rtol=1e-9, atol=1e-9)


def test_error_shrinks_with_eps():
    th = (1.0, 0.3, 1.0)
    x, y, z = _problem(20, th)
    ll_d = DN.loglik(x, y, z, th)[0]
    errs = [abs(TL.loglik(x, y, z, th, nb=80, eps=e)[0] - ll_d) for e in (1e-4, 1e-7, 1e-10)]
    assert errs[2] < errs[0]
    assert errs[2] <= 1e-6 * abs(ll_d)


def test_krige_tlr_matches_dense():
    x, y, z = _problem(16)
    obs, held = inputs.holdout(len(x), 16)
    a = DN.krige(x[obs], y[obs], z[obs], x[held], y[held], TH)
    b = TL.krige(x[obs], y[obs], z[obs], x[held], y[held], TH, nb=60, eps=1e-12)
    np.testing.assert_allclose(b, a, rtol=1e-7, atol=1e-8)
