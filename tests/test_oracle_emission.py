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


@pytest.mark.parametrize("p0,wdt", [(1000.0, 0.05), (5.0, 3.0)])
def test_event_counts_of_the_step_are_poisson_with_mean_W_t(otables, units, p0, wdt):
    # Eq. 6 with the residual-time sub-loop, driven through the real step:
    # electrons gyrating in a uniform B perpendicular to u with the recoil
    # off keep |u| and chi fixed, so each one's emissions over a time t are
    # Poisson(W t), W = C H(chi) / gamma.  The second case has W dt = 3: a
    # wrong residual r of the sub-loop (never decremented, decremented by
    # the optical depth instead of tau / (W dt), ...) changes the law.
    chi = 1.0
    b0 = _b_for_chi(chi, p0, units)
    gam = math.sqrt(1.0 + p0 * p0)
    H = otables.lookup(0, chi)[0]
    W = units.C_rate * H / gam
    dt = wdt / W
    n, n_steps = 3000, 8 if wdt > 1 else 400
    el = _species(n, n, (p0, 0, 0))
    O.init_tau(21, O.ELECTRON, el)
    sim = O.Sim(O.uniform_b_field(b0), _params(dt=dt, seed=21, recoil=0, max_emit=64),
                electrons=el)
    sim.run(n_steps)
    # chi really stayed fixed (|u| conserved by the rotation)
    pm = np.sqrt(el.ux[:n] ** 2 + el.uy[:n] ** 2 + el.uz[:n] ** 2)
    np.testing.assert_allclose(pm, p0, rtol=1e-12)
    np.testing.assert_allclose(el.chi[:n], chi, rtol=1e-10)
    assert sim.stats.n_saturated == 0
    counts = el.nemit[:n].astype(float)
    assert counts.sum() == sim.stats.n_emit
    mean = W * dt * n_steps
    assert counts.mean() == pytest.approx(mean, abs=4 * math.sqrt(mean / n))
    assert counts.var() / counts.mean() == pytest.approx(1.0, abs=0.12)
    # the whole distribution, by chi2 against the Poisson law
    kmax = int(mean + 6 * math.sqrt(mean)) + 1
    kk = np.arange(kmax + 1)
    probs = st.poisson.pmf(kk, mean)
    probs[-1] += st.poisson.sf(kmax, mean)
    obs = np.bincount(np.minimum(counts.astype(int), kmax), minlength=kmax + 1)
    keep = probs * n >= 5  # pool the sparse tails
    e = np.append(probs[keep] * n, probs[~keep].sum() * n)
    o = np.append(obs[keep], obs[~keep].sum())
    chi2 = ((o - e) ** 2 / np.maximum(e, 1e-300)).sum()
    assert st.chi2.sf(chi2, len(e) - 1) > 1e-3


def test_saturated_sub_loop_carries_the_event_to_the_next_step(otables, units):
    # with max_emit = 1 and W dt = 3 most steps reach the cap: the optical
    # depth goes negative and is carried; the event count per step is at
    # most max_emit + nothing else, and saturations are counted
    p0, chi = 5.0, 1.0
    b0 = _b_for_chi(chi, p0, units)
    gam = math.sqrt(1.0 + p0 * p0)
    W = units.C_rate * otables.lookup(0, chi)[0] / gam
    n = 500
    el = _species(n, n, (p0, 0, 0))
    O.init_tau(4, O.ELECTRON, el)
    sim = O.Sim(O.uniform_b_field(b0), _params(dt=3.0 / W, seed=4, recoil=0, max_emit=1),
                electrons=el)
    for step in range(5):
        before = el.nemit[:n].copy()
        sim.run(1)
        assert np.all(el.nemit[:n] - before <= 2)
    assert sim.stats.n_saturated > n
    assert np.any(el.tau[:n] < 0.0)


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


def _uniform_eb(E, B, half=4):
    """A 2D Yee grid with the same float32 value at every node: uniform E, B
    around the origin."""
    n = 2 * half
    comps = [np.full((n, n), v, dtype=np.float32) for v in list(E) + list(B)]
    return O.yee2d_field(comps, 1.0, 1.0, -half, -half)


def _sokolov_expected(units, G, q, dt, E, B, u_half):
    """The continuous step of Eq. 4-5 in the reading of the design notes,
    written out from the equations: f_l = q (E + v x B),
    dv = tau0 (f_l - v (v.f_l)) / (1 + tau0 v.f_l), du = dt (q dv x B - P_rad v),
    dx = dt (v' + dv) with v' from the final momentum."""
    g = math.sqrt(1.0 + u_half @ u_half)
    v = u_half / g
    f = q * (E + np.cross(v, B))
    vf = v @ f
    dv = units.tau0w * (f - v * vf) / (1.0 + units.tau0w * vf)
    prad = units.C_rate * G
    u1 = u_half + dt * (q * np.cross(dv, B) - prad * v)
    g1 = math.sqrt(1.0 + u1 @ u1)
    return u1, dt * (u1 / g1 + dv), dv


@pytest.mark.parametrize("species,q", [(O.ELECTRON, -1.0), (O.POSITRON, 1.0)])
def test_sokolov_delta_v_in_crossed_fields(otables, units, species, q):
    # A generic E and B (neither perpendicular to v nor to each other), so
    # v.f_l != 0 and the denominator 1 + tau0 v.f_l differs from 1 by ~1e-3;
    # gamma ~ 4 and chi ~ 0.5 (the continuous branch forced by chi_th), so
    # the q dv x B force is ~5 % of the momentum change of the step and dv
    # is measured through the position with ~1e-12 relative precision.  A
    # sign error in q dv x B, a dropped denominator or v(v.f_l) term, or a
    # missing +dv in dx/dt fails one of the comparisons.
    F = 6.0e4
    E = np.array([0.3, 0.8, -0.2]) * F
    B = np.array([0.1, -0.4, 0.9]) * F
    field = _uniform_eb(E, B)
    E, B = O.field_eval(field, 0.0, 0.0, 0.0, 0.0)  # the values the step sees
    u0 = np.array([3.0, -2.0, 1.5])
    arr = {"x": [0.0], "y": [0.0], "z": [0.0], "ux": [u0[0]], "uy": [u0[1]], "uz": [u0[2]],
           "w": [1.0]}
    sp = O.Species.from_arrays(arr, 1)
    dt = 1e-6
    kw = dict(electrons=sp) if species == O.ELECTRON else dict(positrons=sp)
    sim = O.Sim(field, _params(dt=dt, chi_th=1e9), **kw)
    sim.run(1)
    assert sim.stats.n_continuous == 1 and sim.stats.n_emit == 0
    u_half = O.boris(q, dt, E, B, u0)
    g_half = math.sqrt(1.0 + u_half @ u_half)
    chi = O.chi_e(E, B, u_half, g_half, units.a_S)
    assert 0.1 < chi < 2.0
    G = otables.lookup(1, chi)[0]
    u1, dx, dv = _sokolov_expected(units, G, q, dt, E, B, u_half)
    got_u = np.array([sp.ux[0], sp.uy[0], sp.uz[0]])
    got_x = np.array([sp.x[0], sp.y[0], sp.z[0]])
    # the size of what is checked
    vf = (u_half / g_half) @ (q * (E + np.cross(u_half / g_half, B)))
    assert abs(units.tau0w * vf) > 1e-4
    dvxb = dt * np.linalg.norm(np.cross(dv, B))
    assert dvxb > 0.02 * np.linalg.norm(u1 - u_half)
    # momentum: the change of the step within 1e-10 of its size
    np.testing.assert_allclose(got_u - u_half, u1 - u_half, rtol=0,
                               atol=1e-10 * np.linalg.norm(u1 - u_half))
    # position: x = dt (v' + dv); dv itself within 1e-8
    g1 = math.sqrt(1.0 + got_u @ got_u)
    dv_got = got_x / dt - got_u / g1
    np.testing.assert_allclose(dv_got, dv, rtol=0, atol=1e-8 * np.linalg.norm(dv))
    np.testing.assert_allclose(got_x, dx, rtol=0, atol=1e-12 * np.linalg.norm(dx))
    # the optical depth does not move in the continuous regime
    assert sp.tau[0] == 0.0


def test_sokolov_step_without_radiation_reaction_is_the_boris_step(units):
    # tau0 -> 0 and P_rad -> 0: the continuous step reduces to the plain
    # Boris step and x += dt v, bit for bit
    E = np.array([2.0e3, -1.0e3, 5.0e2])
    B = np.array([-3.0e2, 4.0e3, 1.0e3])
    field = _uniform_eb(E, B)
    E, B = O.field_eval(field, 0.0, 0.0, 0.0, 0.0)
    u0 = np.array([-1.0, 2.5, 0.5])
    arr = {"x": [0.0], "y": [0.0], "z": [0.0], "ux": [u0[0]], "uy": [u0[1]], "uz": [u0[2]],
           "w": [1.0]}
    sp = O.Species.from_arrays(arr, 1)
    dt = 1e-4
    sim = O.Sim(field, _params(dt=dt, chi_th=1e9), electrons=sp)
    sim.U.tau0w = 0.0
    sim.U.C_rate = 0.0
    sim.run(1)
    u_half = O.boris(-1.0, dt, E, B, u0)
    g = math.sqrt(1.0 + u_half @ u_half)
    assert [sp.ux[0], sp.uy[0], sp.uz[0]] == list(u_half)
    assert [sp.x[0], sp.y[0], sp.z[0]] == list(dt * (u_half / g))


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
