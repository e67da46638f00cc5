"""Matérn covariance (eq. 5, Sec. IV) and its derivatives in theta -- oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

C(r; theta) = theta1 / (2^(theta3-1) Gamma(theta3)) * (r/theta2)^theta3 * K_theta3(r/theta2)
with theta = (sigma^2, beta, nu) = (variance, range, smoothness) and C(0) = sigma^2.

Derivatives (not in the paper; used by the adjoint gradient), x = r / beta,
c_nu = 1 / (2^(nu-1) Gamma(nu)):
  dC/dsigma2 = C / sigma2
  dC/dbeta   = sigma2 c_nu x^(nu+1) K_(nu-1)(x) / beta      [d/dx(x^nu K_nu) = -x^nu K_(nu-1)]
  dC/dnu     = C (ln x - ln 2 - psi(nu)) + sigma2 c_nu x^nu dK_nu/dnu(x)
all three zero at r = 0 except dC/dsigma2 = 1.

K_nu comes from scipy.special.kv.  dK_nu/dnu is taken by Richardson-extrapolated
central differences of kv in the order (two levels, O(h^6)); this is a different
method from the CUDA path's and is pinned by the closed form at nu = 1/2
(DLMF 10.38.7) and by adaptive quadrature of the integral representation
dK_nu/dnu = int_0^inf t sinh(nu t) exp(-x cosh t) dt (DLMF 10.32.9 differentiated).

Pins: tests/test_oracle_matern.py (nu = 1/2 and 3/2 closed forms, nu = 1/2
derivative closed forms, quadrature, finite differences in theta).
"""
from __future__ import annotations

import numpy as np
import scipy.special as sp


def _x_of(r, beta):
    return np.asarray(r, dtype=np.float64) / beta


def c_nu(nu: float) -> float:
    """Normalising constant 1 / (2^(nu-1) Gamma(nu)) of eq. 5."""
    return 1.0 / (2.0 ** (nu - 1.0) * sp.gamma(nu))


def matern(r, sigma2: float, beta: float, nu: float) -> np.ndarray:
    """Eq. 5: C(r; theta), elementwise over the distance array r."""
    x = _x_of(r, beta)
    out = np.full(x.shape, float(sigma2))
    pos = x > 0
    xp = x[pos]
    out[pos] = sigma2 * c_nu(nu) * xp ** nu * sp.kv(nu, xp)
    return out


def dkv_dnu(nu: float, x, h: float = 1e-2) -> np.ndarray:
    """dK_nu(x)/dnu by two-level Richardson extrapolation of central differences."""
    x = np.asarray(x, dtype=np.float64)

    def D(hh):
        return (sp.kv(nu + hh, x) - sp.kv(nu - hh, x)) / (2.0 * hh)

    d1, d2, d4 = D(h), D(h / 2), D(h / 4)
    r1 = (4.0 * d2 - d1) / 3.0      # O(h^4)
    r2 = (4.0 * d4 - d2) / 3.0
    return (16.0 * r2 - r1) / 15.0  # O(h^6)


def matern_derivs(r, sigma2: float, beta: float, nu: float):
    """(dC/dsigma2, dC/dbeta, dC/dnu) elementwise over r."""
    x = _x_of(r, beta)
    C = matern(r, sigma2, beta, nu)
    d_s2 = C / sigma2
    d_b = np.zeros_like(x)
    d_n = np.zeros_like(x)
    pos = x > 0
    xp = x[pos]
    c = c_nu(nu)
    d_b[pos] = sigma2 * c * xp ** (nu + 1.0) * sp.kv(nu - 1.0, xp) / beta
    d_n[pos] = C[pos] * (np.log(xp) - np.log(2.0) - sp.digamma(nu)) \
        + sigma2 * c * xp ** nu * dkv_dnu(nu, xp)
    return d_s2, d_b, d_n
