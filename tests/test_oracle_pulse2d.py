"""Pins of the oracle's 2D Gaussian pulse and its Yee refill (CPU only):
the peak value at the focus, the waist, the intensity FWHM in time, the
2D Gouy phase and amplitude at one Rayleigh length, and the refill at the
focus time against the input generator's snapshot (a separate numpy
implementation)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1311_1107_gb300 import workloads as W

A0, W0, TAU, XF, TF, YA = 200.0, 18.85, 70.7, 120.0, 30.0, 40.0


@pytest.fixture(scope="module")
def p():
    return O.pulse2d(A0, W0, TAU, XF, TF, YA)


def test_peak_at_the_focus(p):
    assert O.pulse2d_eval(p, XF, YA, TF) == A0


def test_waist_at_the_focal_plane(p):
    # at the focus and the envelope peak the phase is 0: E(w0)/E(0) = 1/e
    assert O.pulse2d_eval(p, XF, YA + W0, TF) / A0 == pytest.approx(math.exp(-1.0), rel=1e-14)
    assert O.pulse2d_eval(p, XF, YA - 2 * W0, TF) / A0 == pytest.approx(math.exp(-4.0), rel=1e-14)


def test_intensity_fwhm_in_time(p):
    # on axis at the focus E = a0 env(t) cos(t - t_f): at whole periods the
    # cosine is 1 and E is the envelope; the intensity env^2 is 1/2 at
    # |t - t_f| = tau/2, i.e. env = exp(-2 ln2 (t - t_f)^2 / tau^2)
    for k in (1, 3, 5, 8):
        dt = 2 * math.pi * k
        env = math.exp(-2 * math.log(2) * dt * dt / TAU ** 2)
        assert O.pulse2d_eval(p, XF, YA, TF + dt) == pytest.approx(A0 * env, rel=1e-13)
    half = math.exp(-2 * math.log(2) * (TAU / 2) ** 2 / TAU ** 2) ** 2
    assert half == pytest.approx(0.5, rel=1e-15)


def test_gouy_phase_and_amplitude_of_a_2d_beam(p):
    # one Rayleigh length after the focus, on axis: amplitude a0 2^(-1/4)
    # (a 2D beam spreads in one dimension) and Gouy phase -atan(1)/2 = -pi/8;
    # recovered from the field at the envelope peak and a quarter period
    # before it (where the envelope factor is known)
    zr = 0.5 * W0 * W0
    x = XF + zr
    t0 = TF + zr            # eta = 0
    e0 = O.pulse2d_eval(p, x, YA, t0)
    eq = O.pulse2d_eval(p, x, YA, t0 - math.pi / 2)  # eta = -pi/2
    envq = math.exp(-2 * math.log(2) * (math.pi / 2) ** 2 / TAU ** 2)
    # E(eta=0) = A cos(g), E(eta=-pi/2) = A env cos(pi/2 + g) = -A env sin(g)
    c, s = e0, -eq / envq
    g = math.atan2(s, c)
    assert g == pytest.approx(-math.pi / 8, abs=1e-12)
    assert math.hypot(c, s) == pytest.approx(A0 * 2 ** -0.25, rel=1e-12)


def test_refill_at_the_focus_time_is_the_input_snapshot():
    nx, ny = 96, 48
    dx = dy = W.T_PERIOD / 32.0
    a0, w0, tau = 200.0, W.length(3 * W.LAMBDA_M), W.duration(30e-15)
    xf, ya = 40 * dx, 0.5 * ny * dy
    comps = W.gaussian_2d_snapshot(nx, ny, dx, dy, a0=a0, w0=w0, tau_fwhm=tau, x_focus=xf,
                                   y_axis=ya)
    z = [np.zeros((ny, nx), np.float32) for _ in range(6)]
    f = O.yee2d_field(z, dx, dy)
    O.fill_pulse2d(O.pulse2d(a0, w0, tau, xf, 123.0, ya), f, 123.0)
    for k in (1, 5):
        got, ref = f._keep[k], comps[k]
        ulp = np.spacing(np.abs(ref).astype(np.float32))
        assert np.all(np.abs(got - ref) <= ulp), k
        assert np.abs(ref).max() > 100
    for k in (0, 2, 3, 4):
        assert not f._keep[k].any()
