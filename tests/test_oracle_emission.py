"""Pins of the oracle's Monte-Carlo emission, recoil, pair creation, Sokolov
damping and whole-step bookkeeping (CPU only)."""
import math

import numpy as np
import pytest
import scipy.stats as st

import oracle as O


def _species(n, cap, u, x=None, dims=3, w=1.0):
    arr = {"x": np.zeros(n) if x is None else x, "y": np.arange(n, dtype=float),
           "z": np.zeros(n), "ux": np.full(n, u[0]), "uy": np.full(n, u[1]),
           "uz": np.full(n, u[2]), "w": np.full(n, w)}
    return O.Species.from_arrays(arr, cap, dims)


def _params(**kw):
    p = {"dt": 0.01, "step": 0, "seed": 11, "chi_th": 0.0, "photon_min_gamma": 0.0,
         "pairs": False, "max_emit": 8, "recoil": 1}
    p.update(kw)
    return p


def _b_for_chi(chi, p, units):
    return chi * units.a_S / p


def test_emission_conserves_momentum_and_matches_recoil_energy_defect(units):
    # one electron in a uniform B with chi ~ 2: at every step the Boris
    # momentum equals the final momentum plus the emitted photons (Eq. 8),
    # and the energy change is the analytic defect of collinear recoil.
    p0 = 1000.0
    b0 = _b_for_chi(2.0, p0, units)
    el = _species(1, 1, (p0, 0, 0))
    ph = O.Species(4096)
    O.init_tau(11, O.ELECTRON, el)
    dt = 0.02
    sim = O.Sim(O.uniform_b_field(b0), _params(dt=dt), electrons=el, photons=ph)
    events = 0
    for _ in range(400):
        u_before = np.array([el.ux[0], el.uy[0], el.uz[0]])
        u_b = O.boris(-1.0, dt, [0, 0, 0], [0, 0, b0], u_before)
        n0 = ph.n
        sim.run(1)
        u_after = np.array([el.ux[0], el.uy[0], el.uz[0]])
        k = np.stack([ph.ux[n0:ph.n], ph.uy[n0:ph.n], ph.uz[n0:ph.n]], axis=1)
        np.testing.assert_allclose(u_after + k.sum(axis=0), u_b, rtol=0,
                                   atol=1e-12 * np.linalg.norm(u_b))
        # photons along the electron direction
        for kk in k:
            assert np.linalg.norm(np.cross(kk, u_b)) <= 1e-12 * np.linalg.norm(kk) * np.linalg.norm(u_b)
        # energy defect, emission by emission (photons appended in k order)
        pm = np.linalg.norm(u_b)
        defect = 0.0
        for kk in k:
            gg = np.linalg.norm(kk)
            defect += math.sqrt(1 + (pm - gg) ** 2) + gg - math.sqrt(1 + pm * pm)
            pm -= gg
        de = math.sqrt(1 + u_after @ u_after) + np.linalg.norm(k, axis=1).sum() - math.sqrt(
            1 + u_b @ u_b)
        assert de == pytest.approx(defect, abs=1e-9 * math.sqrt(1 + u_b @ u_b))
        events += ph.n - n0
    assert events > 20


@pytest.mark.parametrize("gam,dt", [(1000.0, 1e-3), (5.0, 2e-2)])
def test_event_counts_are_poisson_with_mean_W_t(otables, units, gam, dt):
    # frozen particle: counts over a time t follow Poisson(W t), W = C H / gamma;
    # the second case has W dt > 1, exercising the residual-time sub-loop.
    chi = 1.0
    H = otables.lookup(0, chi)[0]
    W = units.C_rate * H / gam
    n_steps = int(round(25.0 / (W * dt)))
    sim = O.Sim(O.plane_field(0), {"dt": dt})
    counts = np.array([sim.count_events_frozen(chi, gam, dt, n_steps, seed, max_emit=64)
                       for seed in range(300)])
    mean = W * dt * n_steps
    assert counts.mean() == pytest.approx(mean, abs=4 * math.sqrt(mean / len(counts)))
    assert counts.var() / counts.mean() == pytest.approx(1.0, abs=0.25)


def test_emitted_spectrum_chi2_against_eq2(units):
    # recoil off and uniform B keep chi fixed; the photon fractions
    # u = gamma_gamma / gamma_e must follow the exact CDF of Eq. 7
    chi, p0 = 1.5, 800.0
    b0 = _b_for_chi(chi, p0, units)
    n = 3000
    el = _species(n, n, (p0, 0, 0))
    O.init_tau(5, O.ELECTRON, el)
    ph = O.Species(200000)
    sim = O.Sim(O.uniform_b_field(b0), _params(dt=1e-2, recoil=0, seed=5), electrons=el,
                photons=ph)
    sim.run(60)
    ge = math.sqrt(1 + p0 * p0)
    u = np.sqrt(ph.live("ux") ** 2 + ph.live("uy") ** 2 + ph.live("uz") ** 2) / ge
    assert len(u) > 3000
    edges = np.quantile(u, np.linspace(0, 1, 21))[1:-1]
    cdf = np.array([float(O.cdf_gamma_exact(math.log(e / (1 - e)), chi)) for e in edges])
    probs = np.diff(np.concatenate([[0.0], cdf, [1.0]]))
    obs = np.histogram(u, bins=np.concatenate([[0.0], edges, [1.0]]))[0]
    chi2 = ((obs - probs * len(u)) ** 2 / (probs * len(u))).sum()
    assert st.chi2.sf(chi2, len(probs) - 1) > 1e-3


def test_pair_creation_rate_momentum_and_spectrum(otables, units):
    # photons fixed in a uniform B at chi_gamma = 2: decay fraction 1-exp(-W t);
    # pair momenta add up to the photon's; v = chi_-/chi_gamma follows P_pm
    chi, gg = 2.0, 500.0
    b0 = chi * units.a_S / gg
    n = 4000
    ph = _species(n, n, (gg, 0, 0))
    O.init_tau(9, O.PHOTON, ph)
    el, po = O.Species(n), O.Species(n)
    dt, steps = 0.02, 60
    sim = O.Sim(O.uniform_b_field(b0), _params(dt=dt, pairs=True, seed=9), electrons=el,
                positrons=po, photons=ph)
    vs = []
    for _ in range(steps):
        n0 = el.n
        sim.run(1)
        # pairs created this step: momenta add up to the photon's, v ~ P_pm
        um = np.stack([el.ux[n0:el.n], el.uy[n0:el.n], el.uz[n0:el.n]], 1)
        up = np.stack([po.ux[n0:po.n], po.uy[n0:po.n], po.uz[n0:po.n]], 1)
        np.testing.assert_allclose(um + up, np.tile([gg, 0.0, 0.0], (len(um), 1)), rtol=0,
                                   atol=1e-12 * gg)
        vs.append(np.linalg.norm(um, axis=1) / gg)
    W = units.C_rate * otables.lookup(2, chi)[0] / gg
    frac = np.mean(ph.tau < 0)
    expect = 1 - math.exp(-W * dt * steps)
    assert frac == pytest.approx(expect, abs=4 * math.sqrt(expect * (1 - expect) / n))
    assert el.n == po.n == np.sum(ph.tau < 0)
    v = np.concatenate(vs)
    edges = np.linspace(0.1, 0.9, 9)
    cdf = np.array([float(O.cdf_pair_exact(math.log(e / (1 - e)), chi)) for e in edges])
    probs = np.diff(np.concatenate([[0.0], cdf, [1.0]]))
    obs = np.histogram(v, bins=np.concatenate([[0.0], edges, [1.0]]))[0]
    chi2 = ((obs - probs * len(v)) ** 2 / (probs * len(v))).sum()
    assert st.chi2.sf(chi2, len(probs) - 1) > 1e-3
    # dead photons do not move: their x is where they decayed
    dead = ph.tau < 0
    assert np.all(ph.x[dead] < dt * steps)


def test_sokolov_energy_loss_equals_radiated_power(units):
    # below chi_th the push loses energy at the rate P_rad of Eq. 5 (plus the
    # delta-v x B term, smaller by 1/gamma^2): one step in a uniform B
    p0, chi = 2000.0, 5e-4
    b0 = _b_for_chi(chi, p0, units)
    el = _species(1, 1, (p0, 0, 0))
    O.init_tau(1, O.ELECTRON, el)
    dt = 0.01
    sim = O.Sim(O.uniform_b_field(b0), _params(dt=dt, chi_th=1e-3), electrons=el)
    g0 = math.sqrt(1 + p0 * p0)
    sim.run(1)
    g1 = math.sqrt(1 + el.ux[0] ** 2 + el.uy[0] ** 2 + el.uz[0] ** 2)
    prad = units.C_rate * float(O.G_exact(chi))
    assert (g0 - g1) / dt == pytest.approx(prad, rel=2e-4)
    assert sim.stats.n_emit == 0 and sim.stats.n_continuous == 1
    assert el.tau[0] > 0  # optical depth frozen in the continuous regime


def test_photon_cut_and_subthreshold_energy(units):
    p0 = 50.0
    b0 = _b_for_chi(0.5, p0, units)
    el = _species(200, 200, (p0, 0, 0))
    O.init_tau(2, O.ELECTRON, el)
    ph = O.Species(100000)
    sim = O.Sim(O.uniform_b_field(b0), _params(dt=0.01, photon_min_gamma=2.0, seed=2),
                electrons=el, photons=ph)
    sim.run(100)
    s = sim.stats
    g = np.sqrt(ph.live("ux") ** 2 + ph.live("uy") ** 2 + ph.live("uz") ** 2)
    assert np.all(g > 2.0)
    assert s.n_emit == s.n_photon + s.n_subthreshold and s.n_subthreshold > 0
    assert 0 < s.e_subthreshold <= 2.0 * s.n_subthreshold
