"""Pins of the oracle's RNG, units, fields, Boris push and chi (CPU only)."""
import math

import numpy as np
import pytest

import oracle as O
from tests.conftest import read_golden

ME, QE, C0 = 9.1093837015e-31, 1.602176634e-19, 299792458.0


# ------------------------------------------------------------------ Philox

def test_philox_known_answers():
    kat = read_golden("philox_kat.txt")
    assert len(kat) == 3
    for name, line in kat.items():
        lhs, rhs = line.split(":")
        words = [int(v, 16) for v in lhs.split()]
        expect = [int(v, 16) for v in rhs.split()]
        assert O.philox(words[:4], words[4:6]) == expect, name


def test_u53_range_and_extremes():
    assert O.u53(0, 0) == 2.0 ** -53
    assert O.u53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0
    xs = [O.u53(*O.draw(7, 0, 1, i, 3, 0)[:2]) for i in range(20000)]
    assert 0.0 < min(xs) and max(xs) <= 1.0
    assert np.mean(xs) == pytest.approx(0.5, abs=0.01)


def test_draw_counter_layout():
    # slot -> (ctr0, ctr1), step -> ctr2, species/purpose/k -> ctr3, seed -> key
    seed, slot, step = 0x0123456789ABCDEF, (5 << 32) | 17, 99
    a = O.draw(seed, 2, 3, slot, step, 7)
    b = O.philox([17, 5, 99, (2 << 24) | (3 << 16) | 7], [0x89ABCDEF, 0x01234567])
    assert a == b


# ------------------------------------------------------------------ units

def test_units_against_the_papers_validation_numbers(units):
    g = read_golden("validation_test.txt")
    gamma, b_t = float(g["gamma"]), float(g["b_tesla"])
    b_norm = QE * b_t / (ME * units.omega)
    p = math.sqrt(gamma * gamma - 1)
    chi = O.chi_e([0, 0, 0], [0, 0, b_norm], [p, 0, 0], gamma, units.a_S)
    assert chi == pytest.approx(float(g["chi_e"]), rel=0.03)          # printed "~ 5"
    inv_wb = gamma / (b_norm * units.omega)
    assert inv_wb == pytest.approx(float(g["inv_omega_b_s"]), rel=0.02)
    radius = p / b_norm * C0 / units.omega
    assert radius == pytest.approx(float(g["radius_m"]), rel=0.03)
    es = units.a_S * ME * C0 * units.omega / QE
    assert es == pytest.approx(float(g["e_schwinger"]), rel=0.03)
    assert 1.0 / units.alpha == pytest.approx(float(g["alpha_inv"]), rel=1e-3)


def test_compton_time_and_tau0(units):
    # tau_c = hbar/(m c^2) = 1.2880886e-21 s; tau_0 = 2 r_e / (3 c) = 6.2664e-24 s
    assert units.tau_c == pytest.approx(1.28808867e-21, rel=1e-7)
    assert units.tau0w / units.omega == pytest.approx(6.26642e-24, rel=1e-5)
    # tau_0 = (2/3) alpha tau_c
    assert units.tau0w == pytest.approx(2 / 3 * units.alpha * units.tau_c * units.omega, rel=1e-9)


# ------------------------------------------------------------------ fields

def test_plane_wave_field():
    f = O.plane_field(100.0)
    E, B = O.field_eval(f, 0.3, 1.0, 2.0, 1.1)
    assert E[1] == pytest.approx(100 * math.cos(0.8), rel=1e-15)
    assert B[2] == E[1] and E[0] == E[2] == B[0] == B[1] == 0


def test_gaussian_pulse_shape():
    a0, w0, tau = 50.0, 15.0, 70.0
    f = O.gaussian_field(a0, w0, tau, 3.0, 10.0)
    E, _ = O.field_eval(f, 3.0, 0, 0, 10.0)          # focus, axis, envelope peak
    assert E[1] == pytest.approx(a0, rel=1e-14)
    E, _ = O.field_eval(f, 3.0, w0, 0, 10.0)         # waist radius: 1/e field
    assert E[1] == pytest.approx(a0 / math.e, rel=1e-14)
    E, _ = O.field_eval(f, 3.0, 0, 0, 10.0 + tau / 2)  # half intensity at FWHM/2
    assert E[1] == pytest.approx(a0 / math.sqrt(2) * math.cos(tau / 2), rel=1e-12)
    zr = w0 * w0 / 2                                 # Rayleigh length: a0/sqrt2, Gouy pi/4
    E, B = O.field_eval(f, 3.0 + zr, 0, 0, 10.0 + zr)
    assert E[1] == pytest.approx(a0 / 2, rel=1e-12) and B[2] == E[1]


def test_yee_gather_reproduces_linear_fields():
    nx, ny, dx, dy, x0, y0 = 40, 24, 0.3, 0.25, -1.0, 2.0
    ox = [0.5, 0.0, 0.0, 0.0, 0.5, 0.5]
    oy = [0.0, 0.5, 0.0, 0.5, 0.0, 0.5]
    coef = [(1.0, 0.5, -0.25), (2.0, -0.125, 0.75), (0.5, 0.25, 0.5),
            (-1.0, 0.375, 0.125), (3.0, -0.5, 0.25), (0.25, 0.125, -0.375)]
    comps = []
    for c in range(6):
        X = x0 + (np.arange(nx) + ox[c]) * dx
        Y = y0 + (np.arange(ny) + oy[c]) * dy
        XX, YY = np.meshgrid(X, Y)
        a, b, cc = coef[c]
        comps.append((a + b * XX + cc * YY).astype(np.float32))
    f = O.yee2d_field(comps, dx, dy, x0, y0)
    rng = np.random.default_rng(1)
    for _ in range(50):
        x = x0 + rng.uniform(1.0, nx - 2.0) * dx
        y = y0 + rng.uniform(1.0, ny - 2.0) * dy
        E, B = O.field_eval(f, x, y, 0.0, 0.0)
        got = np.concatenate([E, B])
        want = [a + b * x + cc * y for a, b, cc in coef]
        np.testing.assert_allclose(got, want, rtol=2e-6, atol=2e-6)
    E, B = O.field_eval(f, x0 - 5.0, y0 - 5.0, 0, 0)  # outside: zero field
    assert np.all(E == 0) and np.all(B == 0)


# ------------------------------------------------------------------ Boris

def test_boris_pure_b_conserves_energy_and_rotates_exactly():
    B = np.array([0.0, 0.0, 37.0])
    u = np.array([1500.0, -300.0, 40.0])
    g = math.sqrt(1 + u @ u)
    dt = 0.05
    theta = 2 * math.atan(dt * 37.0 / (2 * g))       # Boris rotation angle per step
    u1 = u.copy()
    for _ in range(1000):
        u1 = O.boris(-1.0, dt, [0, 0, 0], B, u1)
    assert np.linalg.norm(u1) == pytest.approx(np.linalg.norm(u), rel=1e-13)
    assert u1[2] == pytest.approx(u[2], rel=1e-13)
    ang = math.atan2(u1[1], u1[0]) - math.atan2(u[1], u[0])
    expect = (1000 * theta) % (2 * math.pi)            # electron: counter-clockwise about +z
    assert (ang % (2 * math.pi)) == pytest.approx(expect, abs=1e-9)


def test_boris_pure_e_is_exact_impulse():
    E = np.array([3.0, -2.0, 0.5])
    u = np.array([10.0, 1.0, -4.0])
    u1 = O.boris(+1.0, 0.1, E, [0, 0, 0], u)
    np.testing.assert_allclose(u1, u + 0.1 * E, rtol=1e-15, atol=1e-14)


# ------------------------------------------------------------------ chi

def _boost(beta_vec, E, B, four_u):
    """Lorentz boost (c = 1) of fields and a four-momentum (g, u)."""
    bv = np.asarray(beta_vec)
    b2 = bv @ bv
    gb = 1.0 / math.sqrt(1.0 - b2)
    k = gb * gb / (gb + 1.0)
    E, B = np.asarray(E), np.asarray(B)
    E2 = gb * (E + np.cross(bv, B)) - k * bv * (bv @ E)
    B2 = gb * (B - np.cross(bv, E)) - k * bv * (bv @ B)
    g, u = four_u
    n = bv / math.sqrt(b2)
    u2 = u + (gb - 1.0) * (u @ n) * n - gb * bv * g
    g2 = gb * (g - bv @ u)
    return E2, B2, (g2, u2)


def test_chi_e_plane_wave_closed_forms(units):
    a, g = 100.0, 2000.0
    p = math.sqrt(g * g - 1)
    E, B = [0, a, 0], [0, 0, a]
    # head-on: chi = (gamma + |u|) a / a_S ;  co-propagating: (gamma - |u|) a / a_S
    assert O.chi_e(E, B, [-p, 0, 0], g, units.a_S) == pytest.approx((g + p) * a / units.a_S,
                                                                      rel=1e-14)
    assert O.chi_e(E, B, [p, 0, 0], g, units.a_S) == pytest.approx((g - p) * a / units.a_S,
                                                                    rel=1e-6)


def test_chi_e_boost_invariance(units):
    rng = np.random.default_rng(3)
    for _ in range(50):
        E = rng.normal(0, 30, 3)
        B = rng.normal(0, 30, 3)
        u = rng.normal(0, 50, 3)
        g = math.sqrt(1 + u @ u)
        c1 = O.chi_e(E, B, u, g, units.a_S)
        beta = rng.uniform(-0.6, 0.6, 3)
        E2, B2, (g2, u2) = _boost(beta, E, B, (g, u))
        c2 = O.chi_e(E2, B2, u2, g2, units.a_S)
        assert c2 == pytest.approx(c1, rel=1e-9)


def test_chi_gamma_closed_form_and_invariance(units):
    a, gg = 80.0, 300.0
    assert O.chi_gamma([0, a, 0], [0, 0, a], [-gg, 0, 0], units.a_S) == pytest.approx(
        2 * gg * a / units.a_S, rel=1e-14)
    assert O.chi_gamma([0, a, 0], [0, 0, a], [gg, 0, 0], units.a_S) == 0.0
    rng = np.random.default_rng(4)
    for _ in range(50):
        E = rng.normal(0, 30, 3)
        B = rng.normal(0, 30, 3)
        k = rng.normal(0, 1, 3)
        u = 200.0 * k / np.linalg.norm(k)
        c1 = O.chi_gamma(E, B, u, units.a_S)
        E2, B2, (g2, u2) = _boost(rng.uniform(-0.6, 0.6, 3), E, B, (200.0, u))
        assert np.linalg.norm(u2) == pytest.approx(g2, rel=1e-12)
        assert O.chi_gamma(E2, B2, u2, units.a_S) == pytest.approx(c1, rel=1e-9)
