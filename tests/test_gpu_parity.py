"""CUDA path against the CPU oracle, through the C ABI (GPU only).

Bars: event counts and particle indices (slots) bit-exact on the FP64 path;
momenta and energies within 1e-6 relative (FP64) and 1e-4 (mixed); the
mixed path's event decisions may differ from the FP64 oracle only where the
oracle recorded a decision margin below the mixed path's error bound.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_1311_1107_gb300 import qedpic as Q
from paper_1311_1107_gb300 import workloads as W
from paper_1311_1107_gb300.sim import Simulation
from tests.parity import compare_species, oracle_arrays, run_oracle

pytestmark = pytest.mark.gpu

RTOL_FP64 = 1e-6
RTOL_MIXED = 1e-4


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = Q.qp_init_tables(W.LAMBDA_M, 0)
    yield c
    torch.cuda.synchronize()
    Q.qp_destroy(c)


def gpu_run(ctx, workload, n_steps, precision="fp64", chunk=None):
    sim = Simulation(workload, precision=precision, ctx=ctx)
    if chunk:
        done = 0
        while done < n_steps:
            k = min(chunk, n_steps - done)
            sim.run(k)
            done += k
    else:
        sim.run(n_steps)
    torch.cuda.synchronize()
    out = {name: sp.host() for name, sp in sim.species.items()}
    diag = {name: sim.diagnostics(name) for name in sim.species}
    return sim, out, diag


def counters(diag):
    keys = ("n_emit", "n_photon", "n_photon_drop", "n_subthreshold", "n_pair", "n_pair_drop",
            "n_saturated", "n_continuous")
    return {k: sum(getattr(d, k) for d in diag.values()) for k in keys}


def oracle_counters(stats):
    s = stats.as_dict()
    return {k: s[k] for k in ("n_emit", "n_photon", "n_photon_drop", "n_subthreshold", "n_pair",
                              "n_pair_drop", "n_saturated", "n_continuous")}


# ------------------------------------------------------------------ tables, RNG, self-test

def test_tables_match_oracle(ctx):
    t = Q.qp_export_tables(ctx)
    T = O.tables()
    H, Gs, Ts = (np.frombuffer(a, dtype=np.float64) for a in (t.H, t.Gs, t.Ts))
    np.testing.assert_allclose(H, T.H, rtol=1e-11)
    np.testing.assert_allclose(Gs, T.Gs, rtol=1e-11)
    np.testing.assert_allclose(Ts, T.Ts, rtol=1e-11)
    np.testing.assert_allclose(np.frombuffer(t.Cg, dtype=np.float64).reshape(97, 256), T.Cg,
                               rtol=0, atol=1e-12)
    np.testing.assert_allclose(np.frombuffer(t.Cp, dtype=np.float64).reshape(97, 256), T.Cp,
                               rtol=0, atol=1e-12)
    U = O.units(W.LAMBDA_M)
    assert t.a_S == pytest.approx(U.a_S, rel=1e-14)
    assert t.C_rate == pytest.approx(U.C_rate, rel=1e-14)
    assert t.tau0w == pytest.approx(U.tau0w, rel=1e-14)


@pytest.mark.parametrize("n,first", [(1, 0), (1000, 0), (77, 300)])
def test_initial_optical_depth_matches_oracle(ctx, n, first):
    w = W.plane_wave_collision(n=max(n + first, 1))
    sim = Simulation(w, ctx=ctx, load=False)
    el = sim.species["electron"]
    Q.qp_init_optical_depth(ctx, el.handle, 1234, first, n, None)
    torch.cuda.synchronize()
    got = el.t["tau"][first:first + n].cpu().numpy()
    ref = np.zeros(first + n)
    O.lib().or_init_tau(1234, O.ELECTRON, ref.ctypes.data_as(O.C.c_void_p), first, first + n)
    np.testing.assert_allclose(got, ref[first:], rtol=4e-16, atol=0)


def test_bounded_wait_reports_timeout_and_context_survives(ctx):
    assert Q.qp_selftest_wait_timeout(ctx, 2000) == Q.QP_ERR_TIMEOUT
    # the context still steps afterwards
    w = W.plane_wave_collision(n=64, n_steps=5)
    sim, out, diag = gpu_run(ctx, w, 5)
    assert diag["electron"].status == Q.QP_OK
    assert out["electron"]["x"].shape == (64,)


# ------------------------------------------------------------------ FP64 path, full sizes of the small case

def test_plane_wave_collision_full_fp64(ctx):
    """4096 e-, gamma 2000, a0 100, 1000 steps: bit-exact event counts and
    photon slots; momenta within 1e-6."""
    w = W.plane_wave_collision()
    sim, gpu, diag = gpu_run(ctx, w, 1000)
    osim, osp = run_oracle(w, 1000)
    assert counters(diag) == oracle_counters(osim.stats)
    assert sim.live_counts()["photon"] == osp["photon"].n
    e1 = compare_species(gpu["electron"], oracle_arrays(osp["electron"]), RTOL_FP64, 1e-6, "e-")
    e2 = compare_species(gpu["photon"], oracle_arrays(osp["photon"]), RTOL_FP64, 1e-6, "photon")
    assert diag["electron"].status == Q.QP_OK
    print(f"max rel momentum error: electrons {e1:.2e}, photons {e2:.2e}")


def test_plane_wave_ragged_tiles_fp64(ctx):
    """1000 e- (3 full tiles + a ragged tail of 232), 300 steps."""
    w = W.plane_wave_collision(n=1000, n_steps=300)
    sim, gpu, diag = gpu_run(ctx, w, 300, chunk=37)
    osim, osp = run_oracle(w, 300)
    assert counters(diag) == oracle_counters(osim.stats)
    compare_species(gpu["electron"], oracle_arrays(osp["electron"]), RTOL_FP64, 1e-6, "e-")
    compare_species(gpu["photon"], oracle_arrays(osp["photon"]), RTOL_FP64, 1e-6, "photon")


def test_constant_b_cascade_with_pairs_fp64(ctx):
    """The paper's section-4 setting (gamma 3000, B 7.48 MT): electrons,
    photons and pairs, every species appending; 700 e- and 300 seeded
    positrons so both lepton species share the photon chain."""
    w = W.uniform_b_cascade(n=700, n_steps=120, cap=1 << 18)
    rng = np.random.default_rng(5)
    npos = 300
    pos = {"x": rng.normal(0, 1, npos), "y": rng.normal(0, 1, npos), "z": np.zeros(npos),
           "ux": np.zeros(npos), "uy": np.full(npos, 2500.0), "uz": np.zeros(npos),
           "w": np.full(npos, 2.0)}
    tau_p = np.zeros(npos)
    O.lib().or_init_tau(77, O.POSITRON, tau_p.ctypes.data_as(O.C.c_void_p), 0, npos)
    pos["tau"] = tau_p
    sim = Simulation(w, ctx=ctx)
    ps = sim.species["positron"]
    ps.load(pos)
    ps.t["tau"][:npos].copy_(torch.as_tensor(tau_p))
    sim.run(120)
    torch.cuda.synchronize()
    gpu = {name: sp.host() for name, sp in sim.species.items()}
    diag = {name: sim.diagnostics(name) for name in sim.species}
    osim, osp = run_oracle(w, 120, extra={"positron": pos})
    assert counters(diag) == oracle_counters(osim.stats)
    assert osim.stats.n_pair > 10
    for name in ("electron", "positron", "photon"):
        compare_species(gpu[name], oracle_arrays(osp[name]), RTOL_FP64, 1e-6, name)


def test_gaussian_beam_collision_reduced_fp64(ctx):
    """Beam collision geometry (gamma 4000 +-5%, a0 500, 30 fs, waist 2 um)
    with 2000 e- and 200 steps around the peak overlap; pairs on."""
    w = W.beam_collision(n=2000, n_steps=200, buffer=400_000)
    sim, gpu, diag = gpu_run(ctx, w, 200)
    osim, osp = run_oracle(w, 200)
    assert counters(diag) == oracle_counters(osim.stats)
    assert osim.stats.n_emit > 1000
    for name in ("electron", "positron", "photon"):
        compare_species(gpu[name], oracle_arrays(osp[name]), RTOL_FP64, 1e-6, name)


def test_yee_foil_reduced_fp64(ctx):
    """2D laser-on-foil, fixed Yee fields, Sokolov below chi 1e-3: a 256x128
    grid, 4-cell foil (4096 e-), 120 steps."""
    w = W.laser_on_foil(nx=256, ny=128, ppc=8, foil_cells=4, n_steps=120,
                        photon_capacity=1 << 18, pair_capacity=1 << 12)
    sim, gpu, diag = gpu_run(ctx, w, 120)
    osim, osp = run_oracle(w, 120)
    assert counters(diag) == oracle_counters(osim.stats)
    assert osim.stats.n_continuous > 0
    for name in ("electron", "photon"):
        compare_species(gpu[name], oracle_arrays(osp[name]), RTOL_FP64, 1e-6, name)


# ------------------------------------------------------------------ edge cases

def test_photon_overflow_counts_and_keeps_prefix(ctx):
    w = W.plane_wave_collision(n=512, n_steps=200)
    w["capacity"]["photon"] = 3000
    sim, gpu, diag = gpu_run(ctx, w, 200)
    osim, osp = run_oracle(w, 200)
    assert counters(diag) == oracle_counters(osim.stats)
    assert osim.stats.n_photon_drop > 0
    assert sim.live_counts()["photon"] == 3000
    assert diag["electron"].status == Q.QP_WARN_BUFFER_FULL
    compare_species(gpu["photon"], oracle_arrays(osp["photon"]), RTOL_FP64, 1e-6, "photon")
    assert diag["electron"].e_dropped == pytest.approx(osim.stats.e_dropped, rel=1e-9)
    Q.qp_reset_counters(ctx, sim.species["electron"].handle)


def test_saturation_at_max_emissions(ctx):
    w = W.uniform_b_cascade(n=300, n_steps=6, gamma=30.0, cap=1 << 16)
    w["params"]["max_emit"] = 1
    w["params"]["dt"] *= 20
    sim, gpu, diag = gpu_run(ctx, w, 6)
    osim, osp = run_oracle(w, 6)
    assert osim.stats.n_saturated > 0
    assert counters(diag) == oracle_counters(osim.stats)
    compare_species(gpu["electron"], oracle_arrays(osp["electron"]), RTOL_FP64, 1e-6, "e-")


def test_empty_species_and_zero_steps(ctx):
    w = W.plane_wave_collision(n=0, n_steps=3)
    w["electrons"] = {k: np.zeros(0) for k in ("x", "y", "z", "ux", "uy", "uz", "w")}
    w["capacity"] = {"electron": 0, "positron": 0, "photon": 16}
    sim = Simulation(w, ctx=ctx)
    assert sim.run(0) == Q.QP_OK
    sim.run(3)
    torch.cuda.synchronize()
    assert sim.live_counts() == {"electron": 0, "positron": 0, "photon": 0}
    assert sim.diagnostics("photon").status == Q.QP_OK


def test_live_count_above_capacity_is_clamped_and_reported(ctx):
    w = W.plane_wave_collision(n=100, n_steps=2)
    sim = Simulation(w, ctx=ctx)
    sim.species["electron"].n_live.fill_(10_000)   # larger than the 100 slots
    sim.run(2)
    d = sim.diagnostics("electron")
    assert d.status == Q.QP_ERR_INVALID_ARG
    Q.qp_reset_counters(ctx, sim.species["electron"].handle)
    assert sim.diagnostics("electron").status == Q.QP_OK


def test_invalid_step_parameters_rejected_before_enqueue(ctx):
    w = W.plane_wave_collision(n=8, n_steps=1)
    sim = Simulation(w, ctx=ctx)
    for field, value in (("dt", -1.0), ("max_emissions", 0), ("max_emissions", 99),
                         ("precision", 7), ("photon", 9999)):
        p = Q.qp_step_params.from_buffer_copy(sim.params)
        setattr(p, field, value)
        p.n_steps = 1
        with pytest.raises(Q.QPError):
            Q.qp_step(ctx, p, None)


# ------------------------------------------------------------------ determinism, diagnostics

def test_runs_are_bit_identical(ctx):
    w = W.beam_collision(n=3000, n_steps=160, buffer=300_000)
    _, a, _ = gpu_run(ctx, w, 160)
    _, b, _ = gpu_run(ctx, w, 160)
    for name in a:
        for k in a[name]:
            np.testing.assert_array_equal(a[name][k], b[name][k])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_pair_cascade_is_bit_identical_with_many_tiles_per_block(ctx, precision):
    # 20000 electrons in the constant-B cascade: hundreds of thousands of
    # photons, so every block steps many tiles of both chains and carries
    # a pending append from one tile to the next; three runs must agree bit
    # for bit (slot order and counts do not depend on scheduling)
    w = W.uniform_b_cascade(n=20000, n_steps=40, cap=1 << 21)
    runs = []
    for _ in range(3):
        sim = Simulation(w, precision=precision, ctx=ctx)
        assert sim.run(40) >= 0
        torch.cuda.synchronize()
        runs.append({k: sp.host() for k, sp in sim.species.items()})
        d = sim.diagnostics("photon")
        # every pair created is one decay counted by the photon species
        assert runs[-1]["positron"]["x"].shape[0] == d.n_pair - d.n_pair_drop
        sim.close()
    assert runs[0]["photon"]["x"].shape[0] > 500_000
    for r in runs[1:]:
        for name in r:
            for k in r[name]:
                np.testing.assert_array_equal(r[name][k], runs[0][name][k], err_msg=f"{name}.{k}")


def test_diagnostics_match_host_reductions(ctx):
    w = W.beam_collision(n=5000, n_steps=120, buffer=300_000)
    sim, gpu, diag = gpu_run(ctx, w, 120)
    for name in ("electron", "photon"):
        g = gpu[name]
        d = diag[name]
        p2 = g["ux"] ** 2 + g["uy"] ** 2 + g["uz"] ** 2
        alive = g["tau"] >= 0 if name == "photon" else np.ones(len(p2), bool)
        gam = np.sqrt(p2) if name == "photon" else np.sqrt(1 + p2)
        assert d.n_live == len(p2)
        assert d.n_alive == int(alive.sum())
        assert d.energy == pytest.approx(float((g["w"] * gam)[alive].sum()), rel=1e-12)
        assert d.px == pytest.approx(float((g["w"] * g["ux"])[alive].sum()), rel=1e-12, abs=1e-9)
        b = np.clip((np.log10(gam[alive]) + 1.0) * 64 / 6.0, 0, 63).astype(int)
        hist = np.bincount(b, weights=g["w"][alive], minlength=64)
        np.testing.assert_allclose(np.array(d.hist), hist, rtol=1e-12, atol=1e-9)
        d2 = sim.diagnostics(name)
        assert d2.energy == d.energy and list(d2.hist) == list(d.hist)
