"""Pins of oracle/matern.py against closed forms and quadrature (Sec. IV, eq. 5)."""
import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp

from oracle import matern as M

R = np.array([0.0, 1e-9, 1e-4, 0.003, 0.05, 0.2, 0.7, 1.3, 3.0])


@pytest.mark.parametrize("beta", [0.03, 0.1, 0.3])
def test_half_is_exponential(beta):
    # Sec. IV: nu = 1/2 reduces eq. 5 to theta1 exp(-r/theta2)
    got = M.matern(R, 1.7, beta, 0.5)
    np.testing.assert_allclose(got, 1.7 * np.exp(-R / beta), rtol=1e-14, atol=0)


@pytest.mark.parametrize("beta", [0.03, 0.1, 0.3])
def test_three_halves_and_five_halves(beta):
    # K_{3/2}(x) = sqrt(pi/2x) e^-x (1 + 1/x)  =>  C = s2 (1 + x) e^-x
    # K_{5/2}(x) = sqrt(pi/2x) e^-x (1 + 3/x + 3/x^2)  =>  C = s2 (1 + x + x^2/3) e^-x
    x = R / beta
    np.testing.assert_allclose(M.matern(R, 0.8, beta, 1.5), 0.8 * (1 + x) * np.exp(-x), rtol=1e-13)
    np.testing.assert_allclose(M.matern(R, 0.8, beta, 2.5), 0.8 * (1 + x + x * x / 3) * np.exp(-x), rtol=1e-13)


def test_whittle_small_x_limit():
    # nu = 1: x K_1(x) -> 1 as x -> 0 (continuity of C at r = 0)
    got = M.matern(np.array([1e-12, 1e-10]), 1.0, 0.3, 1.0)
    np.testing.assert_allclose(got, 1.0, rtol=1e-9)


def test_dkv_dnu_half_closed_form():
    # DLMF 10.38.7: dK_nu/dnu at nu = 1/2 is sqrt(pi/(2x)) E1(2x) e^x
    x = np.array([1e-3, 0.02, 0.3, 1.0, 4.0, 20.0])
    want = np.sqrt(np.pi / (2 * x)) * sp.exp1(2 * x) * np.exp(x)
    np.testing.assert_allclose(M.dkv_dnu(0.5, x), want, rtol=1e-10)


@pytest.mark.parametrize("nu", [0.3, 1.0, 1.7])
@pytest.mark.parametrize("x", [0.01, 0.4, 2.5, 9.0])
def test_dkv_dnu_quadrature(nu, x):
    # dK_nu/dnu = int_0^inf t sinh(nu t) exp(-x cosh t) dt  (DLMF 10.32.9 differentiated)
    # the integrand is below 1e-300 beyond x cosh t = 700; integrate piecewise up to there
    t_max = np.arccosh(max(700.0 / x, 1.0)) + 1.0
    cuts = np.unique(np.concatenate([[0.0], np.linspace(0.0, t_max, 9)[1:]]))
    val = sum(si.quad(lambda t: t * np.sinh(nu * t) * np.exp(-x * np.cosh(t)), a, b,
                      epsabs=0, epsrel=1e-13, limit=400)[0] for a, b in zip(cuts[:-1], cuts[1:]))
    assert abs(M.dkv_dnu(nu, x) - val) <= 1e-10 * abs(val)


def test_derivs_half_closed_forms():
    s2, beta = 1.3, 0.1
    r = R[R > 0]
    x = r / beta
    d_s2, d_b, d_n = M.matern_derivs(r, s2, beta, 0.5)
    np.testing.assert_allclose(d_s2, np.exp(-x), rtol=1e-14)
    np.testing.assert_allclose(d_b, s2 * np.exp(-x) * r / beta ** 2, rtol=1e-13)
    want_n = s2 * (np.exp(-x) * (np.log(x) + np.log(2) + np.euler_gamma) + np.exp(x) * sp.exp1(2 * x))
    # both forms cancel two O(ln x) terms at tiny x: compare on the sigma^2 scale there
    np.testing.assert_allclose(d_n, want_n, rtol=1e-9, atol=1e-8 * s2)


def test_derivs_zero_at_origin():
    d_s2, d_b, d_n = M.matern_derivs(np.array([0.0]), 2.0, 0.2, 1.3)
    assert d_s2[0] == 1.0 and d_b[0] == 0.0 and d_n[0] == 0.0


@pytest.mark.parametrize("nu", [0.5, 1.0, 1.37])
def test_derivs_finite_difference(nu):
    r = np.array([0.001, 0.02, 0.15, 0.6])
    th = np.array([1.2, 0.17, nu])
    got = M.matern_derivs(r, *th)
    for p in range(3):
        h = 1e-5 * th[p]
        tp, tm = th.copy(), th.copy()
        tp[p] += h
        tm[p] -= h
        fd = (M.matern(r, *tp) - M.matern(r, *tm)) / (2 * h)
        np.testing.assert_allclose(got[p], fd, rtol=1e-7, atol=1e-9)  # FD error ~ h^2, u/h
