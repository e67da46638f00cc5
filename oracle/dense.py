"""Exact dense float64 likelihood, gradient and kriging -- oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* covariance:  Sigma_ij = C(d(s_i, s_j); theta), eq. 5 with Euclidean distance, or the great-circle
               distance of eq. 6 (haversine; x = longitude, y = latitude in degrees, sphere radius r)
               when a radius is given (Sec. IV).
* loglik:      eq. 1, l = -n/2 log(2 pi) - 1/2 log|Sigma| - 1/2 z^T Sigma^{-1} z, through a
               dense Cholesky Sigma = L L^T: log|Sigma| = 2 sum log L_ii, z^T Sigma^{-1} z = ||L^{-1} z||^2.
* loglik_grad: dl/dtheta_p = 1/2 a^T (dSigma/dtheta_p) a - 1/2 tr(Sigma^{-1} dSigma/dtheta_p),
               a = Sigma^{-1} z, with Sigma^{-1} formed explicitly (not in the paper).
* krige:       eq. 4, Z1 = Sigma_12 Sigma_22^{-1} Z2 (zero mean, eq. 3).
* sample:      z = L e, the synthetic measurement generator of Sec. VIII-D.

Pins: tests/test_oracle_dense.py (eigenvalue log-det, n = 1 and n = 2 closed forms,
sigma^2 profile identity, permutation invariance, finite differences, explicit
solve, exact interpolation, great-circle distances along the equator and a meridian,
between the poles and in the small-distance limit).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sl

from . import matern as M


def distances(xa, ya, xb, yb, radius=None) -> np.ndarray:
    """Distance matrix between point sets a and b (Sec. IV): Euclidean, or with a sphere radius the
    great-circle distance of eq. 6, hav(d / r) = hav(phi2 - phi1) + cos(phi1) cos(phi2) hav(lam2 - lam1),
    hav(t) = sin^2(t / 2), for x = longitude lam and y = latitude phi given in degrees."""
    if radius is None:
        return np.hypot(np.subtract.outer(xa, xb), np.subtract.outer(ya, yb))
    la, pa = np.radians(np.asarray(xa, float)), np.radians(np.asarray(ya, float))
    lb, pb = np.radians(np.asarray(xb, float)), np.radians(np.asarray(yb, float))
    hav = lambda t: np.sin(0.5 * t) ** 2
    h = hav(np.subtract.outer(pa, pb)) + np.multiply.outer(np.cos(pa), np.cos(pb)) * hav(np.subtract.outer(la, lb))
    return 2.0 * radius * np.arcsin(np.sqrt(np.clip(h, 0.0, 1.0)))


def covariance(x, y, theta, xb=None, yb=None, radius=None) -> np.ndarray:
    """Sigma(theta) (or the cross-covariance to points (xb, yb))."""
    if xb is None:
        xb, yb = x, y
    return M.matern(distances(x, y, xb, yb, radius), *theta)


def loglik(x, y, z, theta, radius=None):
    """Eq. 1 by dense Cholesky; returns (l, log|Sigma|, z^T Sigma^{-1} z)."""
    n = len(z)
    S = covariance(x, y, theta, radius=radius)
    L = sl.cholesky(S, lower=True)
    logdet = 2.0 * np.sum(np.log(np.diag(L)))
    w = sl.solve_triangular(L, z, lower=True)
    quad = float(w @ w)
    ll = -0.5 * n * np.log(2.0 * np.pi) - 0.5 * logdet - 0.5 * quad
    return ll, logdet, quad


def loglik_grad(x, y, z, theta):
    """(l, grad) with grad = dl/d(sigma^2, beta, nu) via the explicit inverse."""
    n = len(z)
    R = distances(x, y, x, y)
    S = M.matern(R, *theta)
    cf = sl.cho_factor(S, lower=True)
    Sinv = sl.cho_solve(cf, np.eye(n))
    a = sl.cho_solve(cf, z)
    ll, _, _ = loglik(x, y, z, theta)
    grad = np.empty(3)
    for p, G in enumerate(M.matern_derivs(R, *theta)):
        grad[p] = 0.5 * a @ G @ a - 0.5 * np.sum(Sinv * G)
    return ll, grad


def krige(x_obs, y_obs, z_obs, x_new, y_new, theta, radius=None) -> np.ndarray:
    """Eq. 4: Sigma_12 Sigma_22^{-1} z_obs at the new locations."""
    S22 = covariance(x_obs, y_obs, theta, radius=radius)
    S12 = covariance(x_new, y_new, theta, x_obs, y_obs, radius=radius)
    return S12 @ sl.cho_solve(sl.cho_factor(S22, lower=True), z_obs)


def krige_var(x_obs, y_obs, x_new, y_new, theta) -> np.ndarray:
    """Prediction variance of eq. 4's predictor (Sec. III, the conditional covariance
    Sigma_11 - Sigma_12 Sigma_22^{-1} Sigma_21): its diagonal at the new locations."""
    S22 = covariance(x_obs, y_obs, theta)
    S12 = covariance(x_new, y_new, theta, x_obs, y_obs)
    W = sl.solve_triangular(sl.cholesky(S22, lower=True), S12.T, lower=True)
    return theta[0] - np.sum(W * W, axis=0)


def sample(x, y, theta, e, radius=None) -> np.ndarray:
    """z = L e with Sigma(theta) = L L^T (Sec. VIII-D, 'exact computation')."""
    L = sl.cholesky(covariance(x, y, theta, radius=radius), lower=True)
    return L @ e
