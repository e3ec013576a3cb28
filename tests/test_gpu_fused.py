"""Fused steps (qp_step_fused: K steps per launch window, leptons held in
registers; pairs off) against one launch per step (qp_step) and against the
oracle (GPU only).

Both run the same per-particle arithmetic and the same photon motion, and
the fused windows put the new photons in the slot order of separate steps
(a sort on their order keys), so every array of every species must be the
same bits, and every event counter the same number (the sub-threshold
energy is a sum in another order: within 1e-12).  A full photon buffer
drops the same photons unless one window emits more than its capacity."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1311_1107_gb300 import qedpic as Q
from paper_1311_1107_gb300 import workloads as W
from paper_1311_1107_gb300.sim import Simulation
from tests.parity import compare_species, oracle_arrays, run_oracle

pytestmark = pytest.mark.gpu

COUNTERS = ("n_emit", "n_photon", "n_photon_drop", "n_subthreshold", "n_saturated",
            "n_clamped", "n_continuous")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = Q.qp_init_tables(W.LAMBDA_M, 0)
    yield c
    torch.cuda.synchronize()
    Q.qp_destroy(c)


def _no_pairs(w):
    w["params"] = dict(w["params"], pairs=False)
    return w


def _cases():
    return {
        "plane wave": lambda: W.plane_wave_collision(n=1000, n_steps=200),
        "beam": lambda: _no_pairs(W.beam_collision(n=1500, n_steps=200, buffer=300_000)),
        "foil": lambda: _no_pairs(W.laser_on_foil(nx=256, ny=128, ppc=8, foil_cells=4,
                                                  n_steps=200, photon_capacity=1 << 18,
                                                  pair_capacity=1 << 10)),
        "constant B": lambda: _no_pairs(W.uniform_b_cascade(n=700, n_steps=200, cap=1 << 18)),
    }


def _state(sim):
    torch.cuda.synchronize()
    out = {n: sp.host() for n, sp in sim.species.items()}
    diag = {n: sim.diagnostics(n) for n in sim.species}
    return out, diag


def _same(label, a, b, da, db):
    for name in a:
        assert len(a[name]["x"]) == len(b[name]["x"]), (label, name)
        for k, v in a[name].items():
            if v is None:
                continue
            assert np.array_equal(v, b[name][k]), (label, name, k)
    for name in da:
        for c in COUNTERS:
            assert getattr(da[name], c) == getattr(db[name], c), (label, name, c)
        assert da[name].e_subthreshold == pytest.approx(db[name].e_subthreshold, rel=1e-12,
                                                        abs=1e-300)
        assert da[name].status == db[name].status


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", list(_cases()))
def test_fused_windows_give_the_same_bits_as_single_steps(ctx, case, precision):
    w = _cases()[case]()
    n_steps = 200
    ref = Simulation(w, precision=precision, ctx=ctx)
    ref.run(n_steps)
    a, da = _state(ref)
    assert da["electron"].n_emit > 0
    for fuse in (1, 7, 64, n_steps):
        sim = Simulation(w, precision=precision, ctx=ctx)
        sim.run_fused(n_steps, fuse)
        b, db = _state(sim)
        _same(f"{case} {precision} fuse {fuse}", a, b, da, db)
        for sp in list(sim.species.values()):
            Q.qp_destroy_species(ctx, sp.handle)
    print(f"\n[{case} {precision}] {len(a['photon']['x'])} photons, "
          f"{da['electron'].n_emit} emissions: fused = single steps")


@pytest.mark.parametrize("n", [0, 33])
def test_fused_empty_and_ragged_populations(ctx, n):
    # no leptons at all (nothing to step, nothing appended) and two tiles,
    # the second holding one lepton: the same bits as single steps
    w = W.plane_wave_collision(n=n, n_steps=60)
    ref = Simulation(w, precision="mixed", ctx=ctx)
    ref.run(60)
    a, da = _state(ref)
    sim = Simulation(w, precision="mixed", ctx=ctx)
    sim.run_fused(60, 25)
    b, db = _state(sim)
    _same(f"n {n}", a, b, da, db)
    assert len(b["electron"]["x"]) == n
    if n == 0:
        assert len(b["photon"]["x"]) == 0
    for s_ in (ref, sim):
        for sp in list(s_.species.values()):
            Q.qp_destroy_species(ctx, sp.handle)


def test_fused_overflow_drops_the_same_photons(ctx):
    w = W.plane_wave_collision(n=600, n_steps=120)
    w["capacity"] = dict(w["capacity"], photon=3000)
    ref = Simulation(w, precision="fp64", ctx=ctx)
    ref.run(120)
    a, da = _state(ref)
    assert da["electron"].n_photon_drop > 0
    sim = Simulation(w, precision="fp64", ctx=ctx)
    sim.run_fused(120, 50)
    b, db = _state(sim)
    _same("overflow", a, b, da, db)
    assert db["electron"].status == Q.QP_WARN_BUFFER_FULL


def test_fused_window_past_the_capacity_keeps_the_counts(ctx):
    # one window emits more photons than the whole photon capacity: the
    # photons staged first are kept, so which ones survive may differ from
    # single steps; the leptons and every counter may not
    w = W.plane_wave_collision(n=600, n_steps=120)
    w["capacity"] = dict(w["capacity"], photon=500)
    ref = Simulation(w, precision="mixed", ctx=ctx)
    ref.run(120)
    a, da = _state(ref)
    sim = Simulation(w, precision="mixed", ctx=ctx)
    sim.run_fused(120, 120)
    b, db = _state(sim)
    assert da["electron"].n_photon + da["electron"].n_photon_drop > 500
    assert len(b["photon"]["x"]) == len(a["photon"]["x"]) == 500
    for k, v in a["electron"].items():
        assert np.array_equal(v, b["electron"][k]), k
    for c in COUNTERS:
        assert getattr(da["electron"], c) == getattr(db["electron"], c), c
    assert db["electron"].status == Q.QP_WARN_BUFFER_FULL
    assert np.all(b["photon"]["w"] > 0)


def test_fused_plane_wave_against_the_oracle(ctx):
    # the plane-wave case at full size: 4096 e- x 1000 steps, FP64, in
    # windows of 100 steps; events exact, photons slot by slot
    w = W.plane_wave_collision()
    sim = Simulation(w, precision="fp64", ctx=ctx)
    sim.run_fused(1000, 100)
    g, d = _state(sim)
    osim, osp = run_oracle(w, 1000)
    assert d["electron"].n_emit == osim.stats.n_emit
    assert d["electron"].n_photon == osim.stats.n_photon
    compare_species(g["electron"], oracle_arrays(osp["electron"]), 1e-6, 1e-6, "electrons")
    compare_species(g["photon"], oracle_arrays(osp["photon"]), 1e-6, 1e-4, "photons")


def test_fused_rejects_pairs_on(ctx):
    w = W.beam_collision(n=100, n_steps=10, buffer=10_000)
    sim = Simulation(w, precision="fp64", ctx=ctx)
    with pytest.raises(Q.QPError):
        sim.run_fused(10, 5)


@pytest.mark.parametrize("n_steps,fuse", [(10, 0), (70_000, 70_000)])
def test_fused_rejects_bad_windows(ctx, n_steps, fuse):
    # a window of no steps, and one of more than 65535 steps (the steps left
    # to a photon are counted in 16 bits): refused, nothing stepped
    w = W.plane_wave_collision(n=64, n_steps=10)
    sim = Simulation(w, precision="mixed", ctx=ctx)
    before = sim.species["electron"].block.clone()
    with pytest.raises(Q.QPError) as e:
        sim.run_fused(n_steps, fuse)
    assert e.value.status == Q.QP_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert torch.equal(sim.species["electron"].block, before)
    assert sim.step_index == 0


def test_fused_refuses_a_stream_being_captured(ctx):
    # a window reads the lepton counts to the host: during a capture the
    # call returns QP_ERR_INVALID_ARG before anything is enqueued
    w = W.plane_wave_collision(n=100, n_steps=10)
    sim = Simulation(w, precision="mixed", ctx=ctx)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.graph(g, stream=s):
        with pytest.raises(Q.QPError) as e:
            sim.run_fused(10, 5, stream=s)
    assert e.value.status == Q.QP_ERR_INVALID_ARG
    assert sim.run_fused(10, 5) >= 0
    torch.cuda.synchronize()
    assert sim.step_index == 10
