"""Pins of the kinetic-equation solver (Eq. 9-10, oracle/kinetic.py) on the
paper's validation cascade (section 4: gamma 3000 electrons, B = 7.48 MT)."""
import math

import numpy as np
import pytest

import oracle as O
from oracle.kinetic import Cascade
from paper_1311_1107_gb300 import workloads as W

W0 = W.uniform_b_cascade(n=16, n_steps=10)
B0, DT = W0["field"]["b0"], W0["params"]["dt"]
P0 = math.sqrt(3000.0 ** 2 - 1.0)


@pytest.fixture(scope="module")
def kin():
    return Cascade(B0)


def test_rates_equal_the_closed_rates(kin):
    # total emission and pair rates of the quadrature vs C H / gamma, C T / gamma
    C = kin.U.C_rate
    for j in (60, 150, 230, 255):
        exact = C * float(O.H_exact(kin.chi_l[j])) / kin.g[j]
        assert kin.W_emit[j] == pytest.approx(exact, rel=2e-3)
    for k in (180, 260, 300, 315):
        exact = C * float(O.T_exact(kin.chi_k[k])) / kin.k[k]
        assert kin.W_pair[k] == pytest.approx(exact, rel=2e-3)


def test_initial_radiated_power_is_eq5(kin):
    # d(photon energy)/dt at t = 0 for electrons at one momentum = C G(chi)
    j = 240
    N0 = np.zeros(2 * kin.L + kin.G)
    N0[j] = 1.0
    dN = kin.A @ N0
    p_rad = (dN[2 * kin.L:] * kin.k).sum()
    assert p_rad == pytest.approx(kin.U.C_rate * float(O.G_exact(kin.chi_l[j])), rel=2e-3)


def test_lepton_number_conserved_without_pairs():
    k = Cascade(B0, pairs=False, n_lep=120, n_pho=140, n_quad=300)
    N = k.evolve(k.initial_electrons(P0, 1.0), [200 * DT])[0]
    m = k.moments(N)
    assert m["n_electron"] == pytest.approx(1.0, abs=1e-12)
    assert m["n_positron"] == 0.0
    # energy: what the electrons lost is in the photons (deposits conserve
    # momentum, so lepton energy is conserved to the grid's resolution)
    assert m["e_electron"] + m["e_photon"] == pytest.approx(3000.0, rel=2e-3)


def test_kinetic_solution_agrees_with_the_oracle_monte_carlo(kin):
    # 1000 Monte-Carlo electrons: numbers within 6 %, photon energy within 1 %
    from tests.parity import oracle_field
    n = 1000
    w = W.uniform_b_cascade(n=n, n_steps=200, cap=1 << 19)
    el = O.Species.from_arrays(w["electrons"], n + (1 << 19), 3)
    O.init_tau(0, O.ELECTRON, el)
    po, ph = O.Species(1 << 19, 3), O.Species(1 << 21, 3)
    sim = O.Sim(oracle_field(w["field"]), w["params"], electrons=el, positrons=po, photons=ph)
    sim.run(200)
    km = kin.moments(kin.evolve(kin.initial_electrons(P0, 1.0), [200 * DT])[0])
    alive = ph.tau[:ph.n] >= 0
    gg = np.sqrt(ph.ux[:ph.n] ** 2 + ph.uy[:ph.n] ** 2 + ph.uz[:ph.n] ** 2)[alive]
    e_ph = (gg.sum() + sim.stats.e_subthreshold + sim.stats.e_dropped) / n
    assert po.n / n == pytest.approx(km["n_positron"], rel=0.06)
    assert alive.sum() / n == pytest.approx(km["n_photon"], rel=0.06)
    assert e_ph == pytest.approx(km["e_photon"], rel=0.01)
