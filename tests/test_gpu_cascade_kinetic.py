"""The paper's validation test on the GPU (section 4): electrons of energy
3000 m c^2 in a constant 7.48 MT field, photon emission and pair cascade
over three gyrations, against the numerical solution of the kinetic
equations Eq. 9-10 (oracle/kinetic.py).  Numbers, energies and the mean
electron chi of the Monte-Carlo species must follow the kinetic solution
(the comparison the paper makes in its Fig. 1)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.kinetic import Cascade
from paper_1311_1107_gb300 import qedpic as Q
from paper_1311_1107_gb300 import workloads as W
from paper_1311_1107_gb300.sim import Simulation

pytestmark = pytest.mark.gpu

MARKS = (50, 100, 200, 400, 600)
TOL = {"n_electron": 0.03, "n_positron": 0.04, "n_photon": 0.03, "e_electron": 0.05,
       "e_positron": 0.06, "e_photon": 0.01, "chi_electron": 0.06}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = Q.qp_init_tables(W.LAMBDA_M, 0)
    yield c
    torch.cuda.synchronize()
    Q.qp_destroy(c)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_cascade_follows_the_kinetic_equations(ctx, precision):
    n = 1 << 17
    w = W.uniform_b_cascade(n=n, n_steps=600, cap=1 << 20)
    w["capacity"] = {"electron": n + (1 << 20), "positron": 1 << 20, "photon": 1 << 25}
    b0, dt = w["field"]["b0"], w["params"]["dt"]
    kin = Cascade(b0)
    p0 = math.sqrt(3000.0 ** 2 - 1.0)
    kms = [kin.moments(N) for N in kin.evolve(kin.initial_electrons(p0, 1.0),
                                              [m * dt for m in MARKS])]
    sim = Simulation(w, precision=precision, ctx=ctx)
    done = 0
    worst = {}
    for m, km in zip(MARKS, kms):
        assert sim.run(m - done) >= 0
        done = m
        torch.cuda.synchronize()
        d = {k: sim.diagnostics(k) for k in ("electron", "positron", "photon")}
        assert d["photon"].n_photon_drop == 0 and d["electron"].n_photon_drop == 0
        e_sub = d["electron"].e_subthreshold + d["positron"].e_subthreshold
        mc = {"n_electron": d["electron"].n_live / n, "n_positron": d["positron"].n_live / n,
              "n_photon": d["photon"].n_alive / n, "e_electron": d["electron"].energy / n,
              "e_positron": d["positron"].energy / n,
              "e_photon": (d["photon"].energy + e_sub) / n,
              "chi_electron": d["electron"].chi_mean}
        line = " ".join(f"{k} {mc[k]:.4g}/{km[k]:.4g}" for k in mc)
        print(f"\n[{precision} step {m}] MC/kinetic {line}")
        for k in mc:
            rel = abs(mc[k] / km[k] - 1.0)
            worst[k] = max(worst.get(k, 0.0), rel)
            assert rel <= TOL[k], (m, k, mc[k], km[k])
    print(f"[{precision}] largest relative differences: "
          + " ".join(f"{k} {v:.3f}" for k, v in worst.items()))
    sim.close()
