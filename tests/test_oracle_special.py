"""Pins of the oracle's special functions and rate integrals (CPU only).

The oracle evaluates K_nu and int K_1/3 from their integral representation;
these tests hold them against scipy, textbook identities and asymptotic
closed forms, and hold the rate integrals H, G, T (Eq. 2, 3, 5, 6) against
limits derived from the mathematics, a published fit, and independent
adaptive quadrature.
"""
import math

import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp

import oracle as O

XS = np.logspace(-6, math.log10(650.0), 45)


@pytest.mark.parametrize("nu", [1 / 3, 2 / 3, 5 / 3])
def test_bessel_k_matches_scipy(nu):
    k = O.bessel_K(nu, XS)
    ref = sp.kv(nu, XS)
    assert np.max(np.abs(k / ref - 1.0)) < 1e-12


def test_int_k13_matches_adaptive_quadrature():
    xs = XS[::4]
    ik = O.int_K13(xs)
    ref = np.array([si.quad(lambda s: sp.kv(1 / 3, s), x, np.inf, epsabs=0, epsrel=1e-13,
                            limit=500)[0] for x in xs])
    assert np.max(np.abs(ik / ref - 1.0)) < 1e-12


def test_int_k13_at_zero_is_pi_over_sqrt3():
    # int_0^inf K_1/3 = pi / (2 cos(pi/6)) = pi / sqrt(3)
    assert O.int_K13(1e-12) == pytest.approx(math.pi / math.sqrt(3.0), rel=1e-7)


def test_k53_identity():
    # int_x^inf K_5/3 = 2 K_2/3(x) - int_x^inf K_1/3  (from K'_nu recurrences)
    for x in (1e-3, 0.1, 1.0, 5.0, 30.0):
        lhs = si.quad(lambda s: sp.kv(5 / 3, s), x, np.inf, epsabs=0, epsrel=1e-12,
                      limit=500)[0]
        rhs = 2.0 * O.bessel_K(2 / 3, x) - O.int_K13(x)
        assert rhs == pytest.approx(lhs, rel=1e-10)


def synchrotron_function(x):
    """F(x) = x int_x^inf K_5/3, built from the oracle's functions."""
    return x * (2.0 * O.bessel_K(2 / 3, x) - O.int_K13(x))


def test_synchrotron_function_small_x():
    # F(x) -> 4 pi / (sqrt(3) Gamma(1/3)) (x/2)^(1/3) as x -> 0
    for x in (1e-8, 1e-6):
        ref = 4.0 * math.pi / (math.sqrt(3.0) * sp.gamma(1 / 3)) * (x / 2.0) ** (1 / 3)
        assert float(synchrotron_function(x)) == pytest.approx(ref, rel=3e-3)
    # the relative correction shrinks like x^(2/3)
    r1 = float(synchrotron_function(1e-6)) / (4 * math.pi / (math.sqrt(3) * sp.gamma(1 / 3))
                                              * (0.5e-6) ** (1 / 3)) - 1
    r2 = float(synchrotron_function(1e-9)) / (4 * math.pi / (math.sqrt(3) * sp.gamma(1 / 3))
                                              * (0.5e-9) ** (1 / 3)) - 1
    assert abs(r2) < abs(r1) / 50


def test_synchrotron_function_large_x():
    # F(x) -> sqrt(pi x / 2) exp(-x) (1 + 55/(72 x) + ...) as x -> inf
    for x in (50.0, 200.0):
        ref = math.sqrt(math.pi * x / 2.0) * math.exp(-x) * (1.0 + 55.0 / (72.0 * x))
        assert float(synchrotron_function(x)) == pytest.approx(ref, rel=2e-3 * (50.0 / x) ** 2)


def test_photon_spectrum_is_positive():
    # Eq. 2 as printed is negative everywhere; the reading used must give a rate
    for chi in (1e-3, 0.1, 1.0, 10.0):
        u = np.linspace(1e-4, 1 - 1e-4, 101)
        assert np.all(O.F_gamma(u, chi) >= 0.0)


def test_pair_spectrum_positive_and_symmetric():
    for chi in (0.3, 1.0, 10.0):
        v = np.linspace(0.01, 0.49, 25)
        a = O.F_pair(v, chi)
        b = O.F_pair(1.0 - v, chi)
        assert np.all(a > 0.0)
        np.testing.assert_allclose(a, b, rtol=1e-12)


@pytest.mark.parametrize("chi", [1e-5, 1e-4, 1e-3])
def test_H_classical_limit(chi):
    # classical photon number rate: H -> 5 pi chi / 2 (Mellin transform of K_5/3)
    ratio = float(O.H_exact(chi)) / (2.5 * math.pi * chi)
    assert abs(ratio - 1.0) < 2.0 * chi


@pytest.mark.parametrize("chi", [1e-5, 1e-4, 1e-3])
def test_G_larmor_limit(chi, units):
    # Eq. 5 must tend to the Larmor power (2/3) alpha m c^2 chi^2 / tau_c
    prad = units.C_rate * float(O.G_exact(chi))        # in m c^2 omega
    larmor = (2.0 / 3.0) * units.alpha * chi * chi / (units.tau_c * units.omega)
    assert abs(prad / larmor - 1.0) < 10.0 * chi


def test_G_against_published_gaunt_fit():
    # g(chi) = P_quantum / P_classical against the Baier-Katkov fit
    # (1 + 4.8 (1+chi) ln(1+1.7 chi) + 2.44 chi^2)^(-2/3), accurate to a few %
    for chi in (1e-2, 0.1, 0.3, 1.0, 3.0, 10.0, 100.0):
        g = float(O.G_exact(chi)) / (2.0 * math.pi * chi * chi / math.sqrt(3.0))
        fit = (1.0 + 4.8 * (1.0 + chi) * math.log(1.0 + 1.7 * chi) + 2.44 * chi * chi) ** (-2 / 3)
        assert g == pytest.approx(fit, rel=0.025)


def _large_chi_constants():
    B, g23 = sp.beta, sp.gamma(2 / 3)
    pre = 0.5 * g23 * 3 ** (2 / 3)
    cH = pre * (2 * B(1 / 3, 2 / 3) - 2 * B(4 / 3, 2 / 3) + B(7 / 3, 2 / 3))
    cG = pre * (2 * B(4 / 3, 2 / 3) - 2 * B(7 / 3, 2 / 3) + B(10 / 3, 2 / 3))
    cT = pre * (B(2 / 3, 2 / 3) - 2 * B(5 / 3, 5 / 3))
    return cH, cG, cT


def test_large_chi_asymptotes():
    # chi -> inf: K_2/3(z) ~ Gamma(2/3)/2 (2/z)^(2/3) gives H, G, T ~ c chi^(2/3)
    # with Beta-function constants; corrections fall like chi^(-2/3)
    cH, cG, cT = _large_chi_constants()
    # the Ritus constant: total photon rate 1.46 alpha chi^(2/3) / (tau_c gamma)
    assert cH / (math.sqrt(3) * math.pi) == pytest.approx(1.46, abs=0.005)
    prev = None
    for chi in (1e3, 1e4, 1e5):
        dev = np.array([float(O.H_exact(chi)) / (cH * chi ** (2 / 3)) - 1,
                        float(O.G_exact(chi)) / (cG * chi ** (2 / 3)) - 1,
                        float(O.T_exact(chi)) / (cT * chi ** (2 / 3)) - 1])
        assert np.all(np.abs(dev) < 0.02)
        if prev is not None:
            ratio = prev / dev
            np.testing.assert_allclose(ratio, 10 ** (2 / 3), rtol=0.06)
        prev = dev


@pytest.mark.parametrize("chi", [0.01, 0.02, 0.05])
def test_pair_rate_small_chi_law(chi):
    # Laplace method around v = 1/2: T -> 9 pi chi / (16 sqrt 2) exp(-8 / (3 chi))
    ref = 9.0 * math.pi * chi / (16.0 * math.sqrt(2.0)) * math.exp(-8.0 / (3.0 * chi))
    ratio = float(O.T_exact(chi)) / ref
    assert abs(ratio - 1.0) < 0.2 * chi


def _scipy_F_gamma(u, chi):
    z = 2.0 * u / (3.0 * chi * (1.0 - u))
    ik = si.quad(lambda s: sp.kv(1 / 3, s), z, np.inf, epsabs=0, epsrel=1e-12, limit=200)[0]
    return (2.0 + u * u / (1.0 - u)) * sp.kv(2 / 3, z) - ik


def _scipy_F_pair(v, chi):
    z = 2.0 / (3.0 * chi * v * (1.0 - v))
    ik = si.quad(lambda s: sp.kv(1 / 3, s), z, np.inf, epsabs=0, epsrel=1e-12, limit=200)[0]
    return ik + (1.0 / (v * (1.0 - v)) - 2.0) * sp.kv(2 / 3, z)


@pytest.mark.parametrize("chi", [0.05, 1.0, 20.0])
def test_rate_integrals_against_independent_quadrature(chi):
    # brute force: scipy's adaptive quadrature over scipy's Bessel functions
    H = si.quad(lambda u: _scipy_F_gamma(u, chi), 0, 1, epsabs=0, epsrel=1e-10, limit=400,
                points=[min(chi, 0.5)])[0]
    G = si.quad(lambda u: u * _scipy_F_gamma(u, chi), 0, 1, epsabs=0, epsrel=1e-10, limit=400,
                points=[min(chi, 0.5)])[0]
    T = si.quad(lambda v: _scipy_F_pair(v, chi), 0, 1, epsabs=0, epsrel=1e-10, limit=400,
                points=[0.5])[0]
    assert float(O.H_exact(chi)) == pytest.approx(H, rel=1e-8)
    assert float(O.G_exact(chi)) == pytest.approx(G, rel=1e-8)
    if T > 1e-300:
        assert float(O.T_exact(chi)) == pytest.approx(T, rel=1e-8)
