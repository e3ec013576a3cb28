"""Parity at the workloads' full sizes, in the launch configuration the
benchmark times (one qp_step per step, the production species capacities),
checked on sampled particles the oracle follows one by one (GPU only).

Each sampled electron keeps its slot number in the oracle's random streams,
so its trajectory, emissions and recoils are those of the full run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1311_1107_gb300 import qedpic as Q
from paper_1311_1107_gb300 import workloads as W
from paper_1311_1107_gb300.sim import Simulation
from tests.parity import (chaos_aware_compare, distribution_check, head, oracle_arrays,
                          run_oracle)
from tests.test_gpu_mixed import check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = Q.qp_init_tables(W.LAMBDA_M, 0)
    yield c
    torch.cuda.synchronize()
    Q.qp_destroy(c)


def _gpu_steps(ctx, w, precision, n_steps):
    sim = Simulation(w, precision=precision, ctx=ctx)
    for _ in range(n_steps):
        sim.run(1)
    torch.cuda.synchronize()
    el = sim.species["electron"].host()
    diag = {n: sim.diagnostics(n) for n in sim.species}
    counts = sim.live_counts()
    sim.species.clear()
    return el, diag, counts


def _sample(n_all, k, seed=3):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n_all, size=k, replace=False))


def _fp64_check(label, w, n_steps, el, osp, idx):
    """FP64 path vs oracle on sampled electrons, with a twin oracle kicked at
    the rounding level (4e-16 every step; two independent kick patterns) to
    exclude trajectories that amplify
    rounding-level differences past the tolerance over this many steps, and
    decisions closer than 1e-10 excluded (tables built by independent
    quadratures differ at ~1e-14)."""
    n = len(idx)
    o = head(oracle_arrays(osp["electron"]), n)
    g = head(el, n, idx)
    t = []
    for key in (0, 1):
        _, tsp = run_oracle(w, n_steps, sample=idx, noise=4e-16, noise_key=key)
        t.append(head(oracle_arrays(tsp["electron"]), n))
    rep = chaos_aware_compare(g, o, t, 1e-6, label, margin=osp["electron"].margin[:n],
                              margin_min=1e-10, min_comparable=0.5)
    distribution_check(g, o, label + " sampled")
    return rep


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_laser_on_foil_full_size(ctx, precision):
    """131072 e-, 2048x512 grid, all 500 steps; 512 sampled electrons."""
    w = W.laser_on_foil()
    el, diag, counts = _gpu_steps(ctx, w, precision, 500)
    idx = _sample(131072, 512)
    osim, osp = run_oracle(w, 500, sample=idx)
    label = f"foil full size 131072 e- x 500, {precision} (512 sampled)"
    if precision == "fp64":
        _fp64_check(label, w, 500, el, osp, idx)
    else:
        check(label, w, 500, {"electron": el}, osp, osim, None, len(idx), gpu_index=idx,
              sample=idx, min_comparable=0.3)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_beam_collision_full_size_window(ctx, precision):
    """1e7 e- with 1e8-slot photon/pair buffers, the 40 steps that start at
    step 980 (peak overlap at 1000), the beam placed where it would be then;
    256 sampled electrons."""
    w = W.beam_collision()
    start = 980
    w["electrons"]["x"] = w["electrons"]["x"] - start * w["params"]["dt"]
    w["params"]["step"] = start
    el, diag, counts = _gpu_steps(ctx, w, precision, 40)
    assert counts["photon"] > 1_000_000
    idx = _sample(10_000_000, 256)
    osim, osp = run_oracle(w, 40, sample=idx)
    label = f"beam full size 1e7 e- x 40, {precision} (256 sampled)"
    if precision == "fp64":
        _fp64_check(label, w, 40, el, osp, idx)
    else:
        check(label, w, 40, {"electron": el}, osp, osim, None, len(idx), gpu_index=idx,
              sample=idx)
