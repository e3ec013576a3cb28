"""qp_step_host (state held in host memory: copied in, stepped, copied back
in one call) against the same steps on device-resident state (GPU only).

The copies move every FP64 array bit for bit and the step is qp_step's, so
the host blocks after each call must equal the device arrays of a run that
never left the GPU, and the event counters must be the same numbers."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1311_1107_gb300 import qedpic as Q
from paper_1311_1107_gb300 import workloads as W
from paper_1311_1107_gb300.sim import Simulation

pytestmark = pytest.mark.gpu

NAMES = ("electron", "positron", "photon")
COUNTERS = ("n_emit", "n_photon", "n_photon_drop", "n_pair", "n_pair_drop", "n_subthreshold",
            "n_continuous")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = Q.qp_init_tables(W.LAMBDA_M, 0)
    yield c
    torch.cuda.synchronize()
    Q.qp_destroy(c)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["beam with pairs", "foil"])
def test_host_steps_equal_device_steps(ctx, case, precision):
    if case == "foil":
        w = W.laser_on_foil(nx=256, ny=128, ppc=8, foil_cells=4, n_steps=60,
                            photon_capacity=1 << 16, pair_capacity=1 << 10)
    else:
        w = W.beam_collision(n=2000, n_steps=60, buffer=400_000)
    n_steps = 40
    ref = Simulation(w, precision=precision, ctx=ctx)
    ref.run(n_steps)
    torch.cuda.synchronize()

    sim = Simulation(w, precision=precision, ctx=ctx)
    host = {n: torch.empty(sim.species[n].block.shape, dtype=torch.float64, pin_memory=True)
            for n in NAMES}
    counts = sim.live_counts()
    for n in NAMES:
        sim.species[n].copy_state(host[n], counts[n], False)
    torch.cuda.synchronize()
    states = sim.host_states(host, counts)
    for _ in range(n_steps):
        assert sim.run_host(states, 1) >= 0
    got = {n: int(states[k].count) for k, n in enumerate(NAMES)}
    assert got == ref.live_counts()
    if case == "beam with pairs":
        assert got["photon"] > 0 and got["positron"] > 0
    for n in NAMES:
        c = got[n]
        dev = ref.species[n].block[:, :c].cpu().numpy()
        assert np.array_equal(host[n][:, :c].numpy(), dev), (case, precision, n)
    for n in NAMES:
        a, b = ref.diagnostics(n), sim.diagnostics(n)
        for f in COUNTERS:
            assert getattr(a, f) == getattr(b, f), (n, f)
    for s in (ref, sim):
        for sp in list(s.species.values()):
            Q.qp_destroy_species(ctx, sp.handle)


def test_host_step_rejects_a_pitch_below_the_capacity(ctx):
    w = W.plane_wave_collision(n=64, n_steps=4)
    sim = Simulation(w, precision="mixed", ctx=ctx)
    host = {n: torch.empty(sim.species[n].block.shape, dtype=torch.float64, pin_memory=True)
            for n in NAMES}
    states = sim.host_states(host, sim.live_counts())
    states[0].pitch = 8 * (sim.species["electron"].cap - 1)
    with pytest.raises(Q.QPError) as e:
        sim.run_host(states, 1)
    assert e.value.status == Q.QP_ERR_INVALID_ARG
    states[0].pitch = host["electron"].stride(0) * 8
    states[0].count = sim.species["electron"].cap + 1
    with pytest.raises(Q.QPError):
        sim.run_host(states, 1)
    # a step description qp_step rejects: refused before the state is copied
    sim.species["electron"].load(w["electrons"])
    torch.cuda.synchronize()
    before = sim.species["electron"].block.clone()
    states[0].count = 64
    host["electron"].zero_()
    dt = sim.params.dt
    sim.params.dt = -1.0
    with pytest.raises(Q.QPError) as e:
        sim.run_host(states, 1)
    assert e.value.status == Q.QP_ERR_INVALID_ARG
    sim.params.dt = dt
    torch.cuda.synchronize()
    assert torch.equal(sim.species["electron"].block, before)


def test_host_step_with_empty_species_and_zero_steps(ctx):
    w = W.plane_wave_collision(n=0, n_steps=4)
    sim = Simulation(w, precision="fp64", ctx=ctx)
    host = {n: torch.zeros(sim.species[n].block.shape, dtype=torch.float64, pin_memory=True)
            for n in NAMES}
    states = sim.host_states(host, sim.live_counts())
    assert sim.run_host(states, 2) == Q.QP_OK
    assert [int(states[k].count) for k in range(3)] == [0, 0, 0]
    w = W.plane_wave_collision(n=50, n_steps=4)
    sim = Simulation(w, precision="fp64", ctx=ctx)
    host = {n: torch.zeros(sim.species[n].block.shape, dtype=torch.float64, pin_memory=True)
            for n in NAMES}
    counts = sim.live_counts()
    sim.species["electron"].copy_state(host["electron"], counts["electron"], False)
    torch.cuda.synchronize()
    before = host["electron"][:, :50].clone()
    states = sim.host_states(host, counts)
    assert sim.run_host(states, 0) == Q.QP_OK  # no step: the state comes back unchanged
    assert int(states[0].count) == 50
    assert torch.equal(host["electron"][:, :50], before)
