"""Teacher-forced single steps (GPU only): at chosen steps of a run, the
oracle restarts from the CUDA path's own state and both take one step.

This measures the per-step precision of each path independently of how
strongly a trajectory amplifies differences over many steps.  Bars per step:
FP64 path 1e-10 relative (momenta, positions, optical depths; decisions with
a relative margin below 1e-10 excluded), mixed path 1e-5 (margin 1e-4).  Event
counts must agree for every non-marginal particle, and particles appended in
the step are compared slot by slot when no decision was marginal.
"""
import pytest

torch = pytest.importorskip("torch")

from paper_1311_1107_gb300 import qedpic as Q
from paper_1311_1107_gb300 import workloads as W
from paper_1311_1107_gb300.sim import Simulation
from tests.parity import run_oracle_from_state, teacher_forced_compare

pytestmark = pytest.mark.gpu

BARS = {"fp64": (1e-10, 1e-10), "mixed": (1e-5, 1e-4)}  # (rtol, margin_min)

CASES = {
    "plane_wave": (lambda: W.plane_wave_collision(n=2000, n_steps=400), [0, 150, 399]),
    "foil": (lambda: W.laser_on_foil(nx=256, ny=128, ppc=8, foil_cells=4, n_steps=150,
                                     photon_capacity=1 << 18, pair_capacity=1 << 12),
             [0, 60, 149]),
    "beam": (lambda: W.beam_collision(n=2000, n_steps=200, buffer=400_000), [0, 100, 160, 199]),
    "constant_b": (lambda: W.uniform_b_cascade(n=1000, n_steps=100, cap=1 << 18), [0, 40, 99]),
}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = Q.qp_init_tables(W.LAMBDA_M, 0)
    yield c
    torch.cuda.synchronize()
    Q.qp_destroy(c)


def host_state(sim):
    torch.cuda.synchronize()
    return {name: sp.host() for name, sp in sim.species.items()}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", list(CASES))
def test_teacher_forced_step(ctx, case, precision):
    make, steps = CASES[case]
    w = make()
    rtol, margin_min = BARS[precision]
    sim = Simulation(w, precision=precision, ctx=ctx)
    done = 0
    compared = 0
    for k in steps:
        if k > done:
            assert sim.run(k - done) >= 0
            done = k
        before = host_state(sim)
        step_index = sim.step_index
        assert sim.run(1) >= 0
        done += 1
        after = host_state(sim)
        _, osp = run_oracle_from_state(w, before, step_index)
        rep = teacher_forced_compare(before, after, osp, rtol, margin_min,
                                     f"{case} {precision} step {step_index}")
        compared += rep["electron"]["before"]
    assert compared > 0
