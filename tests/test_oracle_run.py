"""Whole-step bookkeeping of the oracle: ordering, capacity, resume,
determinism and degenerate cases (CPU only)."""
import copy
import math

import numpy as np
import pytest

import oracle as O
from paper_1311_1107_gb300 import workloads as W


def _state(sp_list):
    out = []
    for s in sp_list:
        if s is None:
            out.append(None)
            continue
        out.append({nm: None if getattr(s, nm) is None else getattr(s, nm)[:s.n].copy()
                    for nm in O.Species.NAMES})
    return out


def _plane_sim(n=64, steps_cap=64, seed=0, photon_cap=None, a0=100.0):
    w = W.plane_wave_collision(n=n, a0=a0, seed=seed)
    el = O.Species.from_arrays(w["electrons"], n)
    el.x[:n] = np.linspace(0.0, 1.0, n)     # distinct positions identify parents
    O.init_tau(seed, O.ELECTRON, el)
    ph = O.Species(photon_cap or n * steps_cap)
    p = dict(w["params"])
    return O.Sim(O.plane_field(a0), p, electrons=el, photons=ph), el, ph


def test_initial_chi_matches_plane_wave_closed_form(units):
    # head-on: chi = (gamma + |u|) a0 cos(phase) / a_S; 1.213 for gamma 2000, a0 100
    sim, el, ph = _plane_sim(n=4)
    el.x[:4] = 0.0
    sim.run(1)
    g = 2000.0
    # after one Boris step at t = 0 (cos = 1) chi is the head-on value within O(dt)
    assert el.chi[0] == pytest.approx((g + math.sqrt(g * g - 1)) * 100.0 / units.a_S, rel=1e-3)
    assert el.chi[0] == pytest.approx(1.213, abs=1e-3)


def test_photons_appended_in_parent_slot_order():
    sim, el, ph = _plane_sim(n=64)
    for _ in range(30):
        x_before = el.x[:el.n].copy()
        n0 = ph.n
        sim.run(1)
        xs = ph.x[n0:ph.n]
        parents = [int(np.flatnonzero(x_before == v)[0]) for v in xs]
        assert parents == sorted(parents)
        # photon count per parent equals its emissions above the cut (all here)
    assert ph.n > 20


def test_run_is_deterministic_and_resumable():
    a, ea, pa = _plane_sim(n=32)
    b, eb, pb = _plane_sim(n=32)
    a.run(40)
    b.run(20)
    # resume from a copied state in a fresh run object starting at step 20
    ec, pc = copy.deepcopy(eb), copy.deepcopy(pb)
    c = O.Sim(O.plane_field(100.0), {**W.plane_wave_collision()["params"], "step": 20},
              electrons=ec, photons=pc)
    c.run(20)
    b.run(20)
    for x, y in ((_state([ea, pa]), _state([eb, pb])), (_state([ea, pa]), _state([ec, pc]))):
        for sx, sy in zip(x, y):
            for nm in O.Species.NAMES:
                if sx[nm] is not None:
                    np.testing.assert_array_equal(sx[nm], sy[nm])


def test_photon_capacity_overflow_is_counted():
    big, _, phb = _plane_sim(n=64)
    big.run(30)
    total = phb.n
    cap = total // 3
    small, _, phs = _plane_sim(n=64, photon_cap=cap)
    small.run(30)
    assert phs.n == cap
    assert small.stats.n_photon == cap
    assert small.stats.n_photon_drop == total - cap
    # the stored prefix is identical: slots are assigned in the same order
    np.testing.assert_array_equal(phs.ux[:cap], phb.ux[:cap])
    g_drop = np.sqrt(phb.ux[cap:total] ** 2 + phb.uy[cap:total] ** 2 + phb.uz[cap:total] ** 2)
    assert small.stats.e_dropped == pytest.approx(g_drop.sum(), rel=1e-12)


def test_empty_species_and_zero_field():
    el = O.Species(16)
    ph = O.Species(16)
    sim = O.Sim(O.plane_field(100.0), {"dt": 0.1}, electrons=el, photons=ph)
    sim.run(5)
    assert el.n == 0 and ph.n == 0
    el2 = O.Species.from_arrays({"x": np.zeros(3), "y": np.zeros(3), "z": np.zeros(3),
                                 "ux": np.array([5.0, 0, 0]), "uy": np.zeros(3),
                                 "uz": np.zeros(3), "w": np.ones(3)}, 3)
    O.init_tau(0, O.ELECTRON, el2)
    tau0 = el2.tau[:3].copy()
    sim2 = O.Sim(O.plane_field(0.0), {"dt": 0.1}, electrons=el2, photons=ph)
    sim2.run(10)
    np.testing.assert_array_equal(el2.tau[:3], tau0)   # chi = 0: no decrement
    assert el2.x[0] == pytest.approx(10 * 0.1 * 5.0 / math.sqrt(26.0), rel=1e-14)
    assert sim2.stats.n_emit == 0


def test_saturation_carries_optical_depth_to_next_step(units):
    # max_emit = 1 at W dt >> 1: one event per step, the rest carried over
    p0 = 10.0
    b0 = 1.0 * units.a_S / p0
    el = O.Species.from_arrays({"x": np.zeros(1), "y": np.zeros(1), "z": np.zeros(1),
                                "ux": np.array([p0]), "uy": np.zeros(1), "uz": np.zeros(1),
                                "w": np.ones(1)}, 1)
    O.init_tau(0, O.ELECTRON, el)
    ph = O.Species(100)
    sim = O.Sim(O.uniform_b_field(b0), {"dt": 0.5, "max_emit": 1, "photon_min_gamma": 0.0,
                                         "recoil": 0}, electrons=el, photons=ph)
    sim.run(3)
    assert sim.stats.n_saturated == 3
    assert ph.n == 3 and el.tau[0] < 0


def test_pair_capacity_overflow_drops_whole_pairs(units):
    gg, chi = 500.0, 3.0
    b0 = chi * units.a_S / gg
    n = 500
    ph = O.Species.from_arrays({"x": np.zeros(n), "y": np.zeros(n), "z": np.zeros(n),
                                "ux": np.full(n, gg), "uy": np.zeros(n), "uz": np.zeros(n),
                                "w": np.ones(n)}, n)
    O.init_tau(4, O.PHOTON, ph)
    el, po = O.Species(40), O.Species(25)
    sim = O.Sim(O.uniform_b_field(b0), {"dt": 0.05, "pairs": True, "seed": 4},
                electrons=el, positrons=po, photons=ph)
    sim.run(1)
    s = sim.stats
    assert s.n_pair > 25
    assert el.n == 25 and po.n == 25
    assert s.n_pair_drop == s.n_pair - 25


def test_two_dimensional_species_ignore_z():
    w = W.laser_on_foil(nx=64, ny=32, ppc=2, foil_cells=4, n_steps=3)
    el = O.Species.from_arrays(w["electrons"], 1000, dims=2)
    assert el.z is None
    O.init_tau(0, O.ELECTRON, el)
    f = w["field"]
    fld = O.yee2d_field(f["comps"], f["dx"], f["dy"])
    ph = O.Species(10000, dims=2)
    sim = O.Sim(fld, {**w["params"]}, electrons=el, photons=ph)
    sim.run(3)
    assert np.all(np.isfinite(el.live("x"))) and np.all(np.isfinite(el.live("ux")))


def test_restart_from_saved_state_reproduces_the_run():
    # the teacher-forced protocol restarts the oracle from a saved state at a
    # given step; resuming from its own state must reproduce the continuous
    # run bit for bit (all species, appended particles included)
    from paper_1311_1107_gb300 import workloads as W
    from tests.parity import SPECIES, oracle_arrays, run_oracle, run_oracle_from_state
    w = W.uniform_b_cascade(n=64, n_steps=12, cap=1 << 14)
    _, full = run_oracle(w, 12)
    _, part = run_oracle(w, 7)
    state = {name: oracle_arrays(part[name]) for name in SPECIES}
    _, rest = run_oracle_from_state(w, state, 7, n_steps=5)
    for name in SPECIES:
        a, b = oracle_arrays(full[name]), oracle_arrays(rest[name])
        assert len(a["x"]) == len(b["x"])
        for k in ("x", "y", "z", "ux", "uy", "uz", "tau", "w"):
            if a.get(k) is not None:
                assert (a[k] == b[k]).all(), (name, k)
    assert len(oracle_arrays(full["photon"])["x"]) > 0
