"""Spectra and event probabilities of the CUDA path (both precisions) against
the paper's analytic rates (GPU only).

Electrons of one energy perpendicular to a constant B all have the same
chi_e = |u| b0 / a_S (Eq. 1 with E = 0).  In one step:
- the fraction that emits at least once is 1 - exp(-W dt), W = C H(chi)/gamma
  (Eq. 6): a binomial test of the rate;
- the first photon of a particle that emitted exactly once carries
  u = gamma_gamma / gamma_e drawn at that chi: a chi^2 test against the CDF
  of Eq. 2 integrated by quadrature in the oracle (Eq. 7).
Photons of one energy decay into pairs with probability 1 - exp(-W_pm dt),
and v = gamma_-/gamma_gamma follows the CDF of Eq. 3.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
st = pytest.importorskip("scipy.stats")

import oracle as O
from paper_1311_1107_gb300 import qedpic as Q
from paper_1311_1107_gb300 import workloads as W
from paper_1311_1107_gb300.sim import Simulation

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = Q.qp_init_tables(W.LAMBDA_M, 0)
    yield c
    torch.cuda.synchronize()
    Q.qp_destroy(c)


@pytest.fixture(scope="module")
def units():
    return O.units(W.LAMBDA_M)


def chi2_pvalue(x, cdf_at, n_bins=40):
    """chi^2 of the sample x against a CDF, on equiprobable-in-sample bins."""
    edges = np.quantile(x, np.linspace(0, 1, n_bins + 1))[1:-1]
    cdf = np.array([cdf_at(e) for e in edges])
    probs = np.diff(np.concatenate([[0.0], cdf, [1.0]]))
    obs = np.histogram(x, bins=np.concatenate([[0.0], edges, [1.0]]))[0]
    exp = probs * len(x)
    return float(st.chi2.sf(((obs - exp) ** 2 / exp).sum(), n_bins - 1))


def logit(e):
    return math.log(e / (1.0 - e))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("chi", [0.3, 2.0])
def test_emission_probability_and_spectrum(ctx, units, precision, chi):
    n, gamma = 1 << 20, 1500.0
    p0 = math.sqrt(gamma * gamma - 1.0)
    b0 = chi * units.a_S / p0
    H = float(O.H_exact(chi))
    wdt = 0.1
    dt = wdt / (units.C_rate * H / gamma)
    el = {"x": np.zeros(n), "y": np.zeros(n), "z": np.zeros(n), "ux": np.full(n, p0),
          "uy": np.zeros(n), "uz": np.zeros(n), "w": np.ones(n)}
    w = {"name": "spectrum", "dims": 3, "electrons": el,
         "field": {"kind": "uniform_b", "b0": b0},
         "params": {"dt": dt, "seed": 11, "chi_th": 0.0, "photon_min_gamma": 0.0,
                    "pairs": False, "max_emit": 8},
         "capacity": {"electron": n, "positron": 0, "photon": n}}
    sim = Simulation(w, precision=precision, ctx=ctx)
    assert sim.run(1) == 0
    torch.cuda.synchronize()
    e = sim.species["electron"].host()
    ph = sim.species["photon"].host()
    sim.close()
    nemit = e["nemit"].astype(np.int64)
    assert len(ph["x"]) == nemit.sum()  # every photon stored (no energy cut)
    # the push preserves |u| in a pure B field: chi is the same for all
    np.testing.assert_allclose(e["chi"][nemit == 0], chi, rtol=1e-5)
    p_emit = 1.0 - math.exp(-wdt)
    frac = float(np.mean(nemit >= 1))
    assert abs(frac - p_emit) <= 5.0 * math.sqrt(p_emit * (1 - p_emit) / n), (frac, p_emit)
    # first photons of particles with exactly one emission
    first = np.concatenate([[0], np.cumsum(nemit)[:-1]])
    one = nemit == 1
    k = first[one]
    u = np.sqrt(ph["ux"][k] ** 2 + ph["uy"][k] ** 2 + ph["uz"][k] ** 2) / gamma
    assert len(u) > 50_000
    p = chi2_pvalue(u, lambda x: float(O.cdf_gamma_exact(logit(x), chi)))
    print(f"\n[{precision} chi={chi}] emitted fraction {frac:.5f} vs {p_emit:.5f}; "
          f"{len(u)} photons, chi2 p-value {p:.3g}")
    assert p > 1e-3


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pair_probability_and_spectrum(ctx, units, precision):
    n, gg, chi = 1 << 19, 800.0, 3.0
    b0 = chi * units.a_S / gg
    T = float(O.T_exact(chi))
    wdt = 0.2
    dt = wdt / (units.C_rate * T / gg)
    tau = np.zeros(n)
    O.lib().or_init_tau(21, O.PHOTON, tau.ctypes.data_as(O.C.c_void_p), 0, n)
    phot = {"x": np.zeros(n), "y": np.zeros(n), "z": np.zeros(n), "ux": np.full(n, gg),
            "uy": np.zeros(n), "uz": np.zeros(n), "tau": tau, "w": np.ones(n)}
    el0 = {k: np.zeros(0) for k in ("x", "y", "z", "ux", "uy", "uz", "w")}
    w = {"name": "pairs", "dims": 3, "electrons": el0,
         "field": {"kind": "uniform_b", "b0": b0},
         "params": {"dt": dt, "seed": 21, "chi_th": 0.0, "photon_min_gamma": 2.0,
                    "pairs": True, "max_emit": 8},
         "capacity": {"electron": n, "positron": n, "photon": n}}
    sim = Simulation(w, precision=precision, ctx=ctx)
    sim.species["photon"].load(phot)
    assert sim.run(1) == 0
    torch.cuda.synchronize()
    ph = sim.species["photon"].host()
    em = sim.species["electron"].host()
    po = sim.species["positron"].host()
    sim.close()
    dead = ph["tau"] < 0
    assert len(em["x"]) == len(po["x"]) == dead.sum()
    p_pair = 1.0 - math.exp(-wdt)
    frac = float(dead.mean())
    assert abs(frac - p_pair) <= 5.0 * math.sqrt(p_pair * (1 - p_pair) / n), (frac, p_pair)
    # momentum split along k: u_- + u_+ = u_gamma
    np.testing.assert_allclose(em["ux"] + po["ux"], gg, rtol=1e-6 if precision == "mixed" else 1e-12)
    v = em["ux"] / gg
    p = chi2_pvalue(v, lambda x: float(O.cdf_pair_exact(logit(x), chi)))
    print(f"\n[{precision} pairs chi={chi}] decayed fraction {frac:.5f} vs {p_pair:.5f}; "
          f"{len(v)} pairs, chi2 p-value {p:.3g}")
    assert p > 1e-3
