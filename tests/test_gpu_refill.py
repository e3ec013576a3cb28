"""Per-step refill of the foil's 2D Yee grid from the analytic pulse
(qp_fill_yee2d) against the oracle's refill, and the foil stepped with its
fields refilled every step against the oracle doing the same (GPU only).

The library forms each column's factors in FP64 and the nodes in FP32; the
oracle evaluates every node in FP64 and rounds to float.  Bar: every node
within 4e-6 a0.  The refilled fields of the two sides therefore differ at
the 1e-6 level, which the particles carry: the free-running comparison uses
the chaos-aware bar at 1e-4 on both paths (the FP64 path's own 1e-6 bar is
tested on fixed grids, which both sides read identically).  Measured on
GB300: every node within 2.7e-7 a0; comparable electrons within 3.2e-6
(FP64 path) and 8.1e-6 (mixed)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_1311_1107_gb300 import qedpic as Q
from paper_1311_1107_gb300 import workloads as W
from paper_1311_1107_gb300.sim import Simulation, make_field
from tests.parity import (chaos_aware_compare, distribution_check, head, oracle_arrays,
                          oracle_field, oracle_pulse, run_oracle)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = Q.qp_init_tables(W.LAMBDA_M, 0)
    yield c
    torch.cuda.synchronize()
    Q.qp_destroy(c)


@pytest.mark.parametrize("shape", [(2048, 512), (257, 131)])
def test_fill_matches_the_oracle(ctx, shape):
    nx, ny = shape
    w = W.laser_on_foil(nx=nx, ny=ny, ppc=1, foil_cells=2, refill=True, n_steps=500)
    desc = w["field"]
    rf = desc["refill"]
    f, keep = make_field(desc)
    pulse = Q.pulse2d(rf["a0"], rf["w0"], rf["tau_fwhm"], rf["x_focus"], rf["t_focus"],
                      rf["y_axis"])
    of = oracle_field(desc)
    op = oracle_pulse(desc)
    dt = w["params"]["dt"]
    worst = 0.0
    for step in (0, 180, 250, 320, 499):
        t = step * dt
        Q.qp_fill_yee2d(ctx, pulse, f, t)
        torch.cuda.synchronize()
        O.fill_pulse2d(op, of, t)
        for k in (1, 5):
            g = keep[k].cpu().numpy()
            o = of._keep[k]
            err = np.abs(g.astype(np.float64) - o.astype(np.float64)).max() / rf["a0"]
            worst = max(worst, err)
            assert err <= 4e-6, (step, k, err)
        for k in (0, 2, 3, 4):
            assert not keep[k].any()
    print(f"\n[refill {nx}x{ny}] largest node error {worst:.3g} a0")
    assert np.abs(of._keep[1]).max() > 0.5 * rf["a0"]


def test_fill_rejects_bad_arguments(ctx):
    w = W.laser_on_foil(nx=64, ny=32, ppc=1, foil_cells=2, refill=True)
    f, keep = make_field(w["field"])
    p = Q.pulse2d(100.0, 10.0, 50.0, 0.0, 0.0, 0.0)
    bad = Q.qp_field.from_buffer_copy(f)
    bad.kind = Q.QP_FIELD_PLANE
    for grid, pulse in ((bad, p), (f, Q.pulse2d(100.0, 0.0, 50.0, 0.0, 0.0, 0.0))):
        with pytest.raises(Q.QPError):
            Q.qp_fill_yee2d(ctx, pulse, grid, 0.0)


# the refilled fields are FP32 nodes formed differently on the two sides
# (~3e-7 a0 apart): both paths carry that FP32-level difference, so both are
# held to the FP32 (mixed-path) bar
@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-4), ("mixed", 1e-4)])
def test_foil_with_refilled_fields(ctx, precision, rtol):
    n_steps = 150
    w = W.laser_on_foil(nx=256, ny=128, ppc=8, foil_cells=4, n_steps=2 * n_steps,
                        photon_capacity=1 << 18, pair_capacity=1 << 12, refill=True)
    sim = Simulation(w, precision=precision, ctx=ctx)
    sim.run(n_steps)
    torch.cuda.synchronize()
    g = sim.species["electron"].host()
    n = len(w["electrons"]["x"])
    osim, osp = run_oracle(w, n_steps)
    o = head(oracle_arrays(osp["electron"]), n)
    twins = []
    for key in (0, 1):
        # the refilled fields of the two sides differ at FP32 level on both
        # paths: the twins carry FP32-sized kicks
        _, tsp = run_oracle(w, n_steps, noise=2e-7, noise_key=key)
        twins.append(head(oracle_arrays(tsp["electron"]), n))
    rep = chaos_aware_compare(head(g, n), o, twins, rtol, f"foil refilled {precision}",
                              margin=osp["electron"].margin[:n],
                              margin_min=1e-4 if precision == "mixed" else 1e-10,
                              min_comparable=0.05)
    distribution_check(head(g, n), o, f"foil refilled {precision}")
    # the pulse reached the foil: momenta far from thermal
    assert np.abs(o["uy"]).max() > 10.0
    d = sim.diagnostics("electron")
    assert d.n_continuous > 0 and rep["comparable"] > 0
    sim.close()
