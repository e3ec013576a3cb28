"""Pins of the oracle's rate/CDF tables and its inverse-CDF sampler (CPU)."""
import math

import numpy as np
import pytest

import oracle as O


def test_grid_definition(otables):
    T = otables
    assert T.chi[0] == 2.0 ** -14 and T.chi[-1] == 2.0 ** 10
    assert T.chic[0] == 2.0 ** -14 and T.chic[-1] == 2.0 ** 10
    # nodes 2^e (1 + m/32): exactly representable, strictly increasing
    assert np.all(np.diff(T.chi) > 0) and np.all(np.diff(T.chic) > 0)
    assert T.chi[32] == 2.0 ** -13 and T.chi[33] == 2.0 ** -13 * (1 + 1 / 32)
    np.testing.assert_allclose(T.sg, np.linspace(-30, 20, 256), rtol=0, atol=1e-13)
    np.testing.assert_allclose(T.sp, np.linspace(-20, 20, 256), rtol=0, atol=1e-13)


def test_rate_tables_match_exact_at_nodes(otables):
    T = otables
    idx = [0, 100, 192, 400, 500, 700, 768]
    for j in idx:
        c = T.chi[j]
        assert T.H[j] == pytest.approx(float(O.H_exact(c)), rel=1e-13)
        assert T.Gs[j] * c == pytest.approx(float(O.G_exact(c)), rel=1e-13)
        if c >= 2.0 ** -8:
            assert T.Ts[j] * math.exp(-8 / (3 * c)) == pytest.approx(float(O.T_exact(c)),
                                                                      rel=1e-12)
        else:
            assert T.Ts[j] == 0.0


@pytest.mark.parametrize("which,exact,lo", [(0, O.H_exact, 0.0), (1, O.G_exact, 0.0),
                                            (2, O.T_exact, 2.0 ** -8)])
def test_rate_interpolation_error_bound(otables, which, exact, lo):
    # linear interpolation of the scaled tables on the 32-per-octave grid:
    # stated bound 1e-4 relative at every octave position
    T = otables
    worst = 0.0
    for j in range(3, 768, 29):
        for frac in (0.25, 0.5, 0.75):
            c = T.chi[j] + frac * (T.chi[j + 1] - T.chi[j])
            if c < lo:
                continue
            v, cl = T.lookup(which, c)
            assert not cl
            worst = max(worst, abs(v / float(exact(c)) - 1.0))
    assert worst < 1e-4


def test_rate_lookup_below_and_above_range(otables):
    T = otables
    chi = 1e-6
    assert T.lookup(0, chi)[0] == pytest.approx(2.5 * math.pi * chi, rel=1e-15)
    assert T.lookup(1, chi)[0] == pytest.approx(2 * math.pi * chi * chi / math.sqrt(3), rel=1e-15)
    assert T.lookup(2, chi)[0] == 0.0
    assert T.lookup(2, 2.0 ** -8 * 0.999)[0] == 0.0
    v, cl = T.lookup(0, 5000.0)
    assert cl and v == T.H[-1]


def test_cdf_rows_monotone_and_normalised(otables):
    T = otables
    assert np.all(np.diff(T.Cg, axis=1) >= 0)
    assert np.all(np.diff(T.Cp, axis=1) >= 0)
    assert np.all(T.Cg[:, -1] <= 1.0) and np.all(T.Cg[:, -1] > 1 - 1e-12)
    rows = T.Cp[T.chic > 0.02]
    assert np.all(rows[:, -1] > 1 - 1e-12)
    # pair rows are symmetric in v <-> 1 - v
    good = T.chic > 0.05
    np.testing.assert_allclose(T.Cp[good], 1.0 - T.Cp[good][:, ::-1], atol=1e-10)


def test_cdf_rows_match_exact(otables):
    T = otables
    for j in (10, 48, 70, 90):
        for i in (40, 120, 200):
            assert T.Cg[j, i] == pytest.approx(float(O.cdf_gamma_exact(T.sg[i], T.chic[j])),
                                               rel=1e-11, abs=1e-15)


def _stratified(n):
    return (np.arange(n) + 0.5) / n


@pytest.mark.parametrize("chi", [1e-3, 0.1, 1.0, 10.0])
def test_sampler_reproduces_exact_cdf(otables, chi):
    # Eq. 7 inverted on the tables: the empirical CDF of samples drawn at
    # stratified xi' must follow the exact CDF within the table error.
    n = 4000
    xs = _stratified(n)
    u = np.array([otables.sample_gamma(chi, x) for x in xs])
    assert np.all(np.diff(u) >= 0) and np.all((u > 0) & (u < 1))
    qs = np.quantile(u, [0.05, 0.25, 0.5, 0.75, 0.95])
    for q, target in zip(qs, [0.05, 0.25, 0.5, 0.75, 0.95]):
        s = math.log(q / (1 - q))
        assert float(O.cdf_gamma_exact(s, chi)) == pytest.approx(target, abs=3e-3)


def test_sampler_power_tail(otables):
    # below the first u-node the CDF follows u^(1/3): u = u0 (xi/C0)^3
    chi = 1.0
    j = int(np.searchsorted(otables.chic, chi, side="right") - 1)
    assert otables.chic[j] == chi
    c0 = otables.Cg[j, 0]
    xi = 0.25 * c0
    u = otables.sample_gamma(chi, xi)
    assert u == pytest.approx(otables.ug[0] * 0.25 ** 3, rel=1e-12)


def test_sampler_scales_below_grid(otables):
    # classical regime: the spectrum in u scales with chi
    chi0 = otables.chic[0]
    a = otables.sample_gamma(chi0, 0.37)
    b = otables.sample_gamma(chi0 / 8, 0.37)
    assert b == pytest.approx(a / 8, rel=1e-14)


@pytest.mark.parametrize("chi", [0.5, 2.0, 20.0])
def test_pair_sampler_reproduces_exact_cdf(otables, chi):
    n = 4000
    v = np.array([otables.sample_pair(chi, x) for x in _stratified(n)])
    assert np.all(np.diff(v) >= 0) and np.all((v > 0) & (v < 1))
    # symmetric spectrum: median 1/2, quantiles mirror each other
    assert np.median(v) == pytest.approx(0.5, abs=2e-3)
    q = np.quantile(v, [0.1, 0.9])
    assert q[0] == pytest.approx(1 - q[1], abs=3e-3)
    for qq, target in zip(np.quantile(v, [0.1, 0.3]), [0.1, 0.3]):
        s = math.log(qq / (1 - qq))
        assert float(O.cdf_pair_exact(s, chi)) == pytest.approx(target, abs=3e-3)
