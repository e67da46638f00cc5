"""Pins of oracle/dense.py: eq. 1 likelihood, gradient and eq. 4 kriging."""
import numpy as np
import pytest

from oracle import dense as DN
from oracle import matern as M
from paper_1804_09137_gb300 import inputs

TH = (1.0, 0.1, 0.5)


def _problem(side, theta=TH):
    x, y = inputs.jittered_grid(side)
    z = DN.sample(x, y, theta, inputs.standard_normal(len(x)))
    return x, y, z


def test_logdet_eigenvalues():
    x, y, z = _problem(12, (1.0, 0.3, 1.0))
    ll, ld, q = DN.loglik(x, y, z, (1.0, 0.3, 1.0))
    lam = np.linalg.eigvalsh(DN.covariance(x, y, (1.0, 0.3, 1.0)))
    assert abs(ld - np.sum(np.log(lam))) <= 1e-9 * abs(ld)
    assert abs(q - np.sum((np.linalg.eigh(DN.covariance(x, y, (1.0, 0.3, 1.0)))[1].T @ z) ** 2 / lam)) <= 1e-8 * q


def test_single_point_closed_form():
    ll, ld, q = DN.loglik(np.array([0.3]), np.array([0.4]), np.array([1.7]), (2.5, 0.1, 0.8))
    want = -0.5 * np.log(2 * np.pi) - 0.5 * np.log(2.5) - 1.7 ** 2 / (2 * 2.5)
    assert abs(ll - want) < 1e-15 * abs(want) + 1e-15


def test_two_points_by_hand():
    th = (1.4, 0.2, 0.5)
    x, y, z = np.array([0.1, 0.4]), np.array([0.2, 0.6]), np.array([0.7, -1.1])
    c = 1.4 * np.exp(-0.5 / 0.2)  # distance 0.5, exponential model
    det = 1.4 ** 2 - c ** 2
    quad = (1.4 * z[0] ** 2 - 2 * c * z[0] * z[1] + 1.4 * z[1] ** 2) / det
    want = -np.log(2 * np.pi) - 0.5 * np.log(det) - 0.5 * quad
    ll, ld, q = DN.loglik(x, y, z, th)
    assert abs(ll - want) <= 1e-14 * abs(want)


def test_sigma2_profile_identity():
    # Sigma = sigma2 R and q = z^T Sigma^{-1} z  =>  dl/dsigma2 = (q - n) / (2 sigma2)
    x, y, z = _problem(8)
    th = (1.7, 0.1, 0.5)
    ll, g = DN.loglik_grad(x, y, z, th)
    _, _, q = DN.loglik(x, y, z, th)
    assert abs(g[0] - (q - len(z)) / (2 * th[0])) <= 1e-10 * abs(g[0]) + 1e-10


def test_permutation_invariance():
    x, y, z = _problem(10)
    p = np.random.default_rng(5).permutation(len(x))
    a = DN.loglik(x, y, z, TH)[0]
    b = DN.loglik(x[p], y[p], z[p], TH)[0]
    assert abs(a - b) <= 1e-12 * abs(a)


@pytest.mark.parametrize("theta", [(1.0, 0.1, 0.5), (1.0, 0.3, 1.0), (0.8, 0.05, 1.4)])
def test_gradient_central_differences(theta):
    x, y, z = _problem(8, theta)
    _, g = DN.loglik_grad(x, y, z, theta)
    th = np.array(theta)
    for p in range(3):
        h = 1e-6 * th[p]
        tp, tm = th.copy(), th.copy()
        tp[p] += h
        tm[p] -= h
        fd = (DN.loglik(x, y, z, tp)[0] - DN.loglik(x, y, z, tm)[0]) / (2 * h)
        assert abs(g[p] - fd) <= 1e-5 * max(abs(fd), 1.0), (p, g[p], fd)


def test_gradient_trace_term_dropped_would_fail():
    # the trace term matters: a^T G a / 2 alone differs from the full gradient
    x, y, z = _problem(8)
    _, g = DN.loglik_grad(x, y, z, TH)
    S = DN.covariance(x, y, TH)
    a = np.linalg.solve(S, z)
    G = M.matern_derivs(DN.distances(x, y, x, y), *TH)[1]
    assert abs(0.5 * a @ G @ a - g[1]) > 1e-3 * abs(g[1])


def test_krige_explicit_solve_and_interpolation():
    x, y, z = _problem(14)
    obs, held = inputs.holdout(len(x), 20)
    zp = DN.krige(x[obs], y[obs], z[obs], x[held], y[held], TH)
    S = DN.covariance(x, y, TH)
    want = S[np.ix_(held, obs)] @ np.linalg.solve(S[np.ix_(obs, obs)], z[obs])
    np.testing.assert_allclose(zp, want, rtol=1e-9, atol=1e-11)
    # exact interpolator without a nugget: predicting at observed points returns z
    zi = DN.krige(x[obs], y[obs], z[obs], x[obs[:5]], y[obs[:5]], TH)
    np.testing.assert_allclose(zi, z[obs[:5]], atol=1e-8)


def test_sample_covariance_factor():
    x, y = inputs.jittered_grid(6)
    S = DN.covariance(x, y, TH)
    E = np.eye(len(x))
    Z = np.stack([DN.sample(x, y, TH, E[:, i]) for i in range(len(x))], axis=1)  # = L
    np.testing.assert_allclose(Z @ Z.T, S, atol=1e-13)
    assert np.allclose(np.triu(Z, 1), 0)


def test_krige_var_one_and_two_points_by_hand():
    """Conditional variance sigma2 - c^T K^{-1} c written out for one and two observed points (nu = 1/2:
    C(r) = sigma2 exp(-r / beta))."""
    s2, be = 1.7, 0.2
    th = (s2, be, 0.5)
    xo, yo = np.array([0.1]), np.array([0.2])
    xn, yn = np.array([0.25]), np.array([0.1])
    r = np.hypot(0.15, -0.1)
    c = s2 * np.exp(-r / be)
    assert abs(DN.krige_var(xo, yo, xn, yn, th)[0] - (s2 - c * c / s2)) <= 1e-14
    xo2, yo2 = np.array([0.1, 0.4]), np.array([0.2, 0.3])
    k12 = s2 * np.exp(-np.hypot(0.3, 0.1) / be)
    c1 = s2 * np.exp(-np.hypot(0.15, -0.1) / be)
    c2 = s2 * np.exp(-np.hypot(-0.15, -0.2) / be)
    det = s2 * s2 - k12 * k12
    quad = (s2 * c1 * c1 - 2 * k12 * c1 * c2 + s2 * c2 * c2) / det
    assert abs(DN.krige_var(xo2, yo2, xn, yn, th)[0] - (s2 - quad)) <= 1e-13


def test_krige_var_interpolation_far_field_and_bounds():
    """Zero at an observed location (no nugget), sigma2 far from every observation, inside [0, sigma2]."""
    x, y, _ = _problem(12)
    obs, held = inputs.holdout(len(x), 20)
    v_obs = DN.krige_var(x[obs], y[obs], x[obs[:5]], y[obs[:5]], TH)
    assert np.all(np.abs(v_obs) <= 1e-8)
    v_far = DN.krige_var(x[obs], y[obs], np.array([60.0]), np.array([60.0]), TH)
    assert abs(v_far[0] - TH[0]) <= 1e-12
    v = DN.krige_var(x[obs], y[obs], x[held], y[held], TH)
    assert np.all(v >= -1e-10) and np.all(v <= TH[0] + 1e-12)


def test_great_circle_distance_closed_cases():
    """Eq. 6 against distances known without the haversine: arcs along the equator and along a
    meridian, pole to pole, symmetry, and the small-distance limit r sqrt(dphi^2 + cos^2 phi dlam^2)."""
    r = 6371.0
    d = DN.distances(np.array([10.0]), np.array([0.0]), np.array([55.0]), np.array([0.0]), r)[0, 0]
    assert abs(d - r * np.radians(45.0)) <= 1e-9 * r
    d = DN.distances(np.array([-20.0]), np.array([-30.0]), np.array([-20.0]), np.array([40.0]), r)[0, 0]
    assert abs(d - r * np.radians(70.0)) <= 1e-9 * r
    d = DN.distances(np.array([0.0]), np.array([90.0]), np.array([123.0]), np.array([-90.0]), r)[0, 0]
    assert abs(d - np.pi * r) <= 1e-9 * r
    xa, ya = np.array([3.0, -70.0, 120.0]), np.array([10.0, 45.0, -60.0])
    D = DN.distances(xa, ya, xa, ya, r)
    assert np.allclose(D, D.T, rtol=0, atol=1e-9) and np.all(np.abs(np.diag(D)) <= 1e-9)
    phi, dphi, dlam = np.radians(50.0), np.radians(1e-3), np.radians(2e-3)
    d = DN.distances(np.array([7.0]), np.array([50.0]), np.array([7.002]), np.array([50.001]), 1.0)[0, 0]
    approx = np.sqrt(dphi ** 2 + (np.cos(phi) * dlam) ** 2)
    assert abs(d - approx) <= 1e-5 * approx
