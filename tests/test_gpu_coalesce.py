"""Super-photon compaction and coalescence on the GPU (qp_compact_photons,
qp_coalesce_photons) against the oracle, through the C ABI (GPU only).

The oracle and the library form the same groups (exact FP64 decisions and
bit extractions), sum them in slot order with the same operations, and
write the survivors in slot order: slots, weights, positions and momenta
must agree bit for bit, the fresh optical depths within the last bit of a
logarithm.  Cases: random populations with decayed photons, groups of every
size, 2D and 3D, counts that fill several blocks with a ragged end, empty
and single-photon species; photons of a real cascade; and a cascade
compacted and coalesced every few steps, against the oracle doing the same
and against the kinetic equations."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_1311_1107_gb300 import qedpic as Q
from paper_1311_1107_gb300 import workloads as W
from paper_1311_1107_gb300.sim import DeviceSpecies, Simulation
from tests.parity import momentum_error, oracle_arrays, position_error, run_oracle_from_state

pytestmark = pytest.mark.gpu

KEYS = ("x", "y", "z", "ux", "uy", "uz", "w")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = Q.qp_init_tables(W.LAMBDA_M, 0)
    yield c
    torch.cuda.synchronize()
    Q.qp_destroy(c)


def _random(n, seed, dims=3, dead=0.2, spread=0.15, lo=3.0, hi=3000.0):
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n, 3)) * spread + [1.0, 0.0, 0.0]
    d /= np.linalg.norm(d, axis=1)[:, None]
    e = np.exp(rng.uniform(np.log(lo), np.log(hi), n))
    arr = {"x": rng.uniform(0, 8, n), "y": rng.uniform(0, 8, n),
           "z": rng.uniform(0, 8, n) if dims == 3 else np.zeros(n),
           "ux": e * d[:, 0], "uy": e * d[:, 1], "uz": e * d[:, 2] if dims == 3 else e * d[:, 2],
           "w": rng.uniform(0.5, 2.0, n),
           "tau": np.where(rng.uniform(size=n) < dead, -1.0, rng.exponential(size=n)),
           "chi": rng.uniform(0, 1, n), "nemit": (rng.uniform(size=n) < 0.1).astype(np.int32)}
    return arr


def _gpu(ctx, arr, cap, dims):
    n = len(arr["x"])
    sp = DeviceSpecies(ctx, Q.QP_PHOTON, cap, dims)
    sp.load(arr, n)
    if n:
        sp.chi[:n].copy_(torch.as_tensor(arr["chi"]))
        sp.nemit[:n].copy_(torch.as_tensor(arr["nemit"]))
    return sp


def _oracle(arr, cap, dims):
    n = len(arr["x"])
    sp = O.Species.from_arrays(arr, max(cap, 1), dims)
    sp.tau[:n] = arr["tau"]
    sp.chi[:n] = arr["chi"]
    sp.nemit[:n] = arr["nemit"]
    return sp


def _compare(label, g, o, dims, n):
    assert len(g["x"]) == n == o.n, (label, len(g["x"]), o.n)
    for k in KEYS:
        if k == "z" and dims == 2:
            continue
        np.testing.assert_array_equal(g[k], getattr(o, k)[:n], err_msg=f"{label} {k}")
    np.testing.assert_allclose(g["tau"], o.tau[:n], rtol=4e-16, atol=0, err_msg=label)
    np.testing.assert_array_equal(g["chi"], o.chi[:n])
    np.testing.assert_array_equal(g["nemit"], o.nemit[:n])


PARAMS = dict(box=(0.0, 0.0, 0.0, 2.0, 2.0, 2.0), cells=(4, 4, 4))


@pytest.mark.parametrize("dims", [3, 2])
@pytest.mark.parametrize("n,eb,db,m,mg", [(0, 8, 8, 3, 0), (1, 8, 8, 3, 0), (777, 2, 2, 3, 0),
                                          (200_003, 4, 4, 3, 0), (200_003, 1, 1, 50, 0),
                                          (200_003, 1, 1, 3, 7), (50_000, 1, 1, 3, 100_000)])
def test_coalescence_matches_the_oracle(ctx, dims, n, eb, db, m, mg):
    arr = _random(n, n + dims, dims)
    cap = n + 5
    cells = PARAMS["cells"] if dims == 3 else (4, 4, 1)
    g = _gpu(ctx, arr, cap, dims)
    o = _oracle(arr, cap, dims)
    p = Q.coalesce_params(PARAMS["box"], cells, eb, db, m, seed=3, step=17, max_group=mg)
    st = Q.qp_coalesce_photons(ctx, g.handle, p)
    so = O.coalesce(o, O.coalesce_params(PARAMS["box"], cells, eb, db, m, dims=dims, seed=3,
                                         step=17, max_group=mg))
    print(f"\n[coalesce dims {dims} n {n}] gpu {st} oracle {so}")
    assert st["groups_merged"] == so["groups_merged"]
    assert st["photons_merged"] == so["photons_merged"]
    assert st["n_before"] == n and st["n_after"] == so["n_after"] == g.count()
    _compare(f"coalesce {dims}D n={n}", g.host(), o, dims, so["n_after"])
    Q.qp_destroy_species(ctx, g.handle)


@pytest.mark.parametrize("n", [0, 1, 129, 300_001])
def test_compaction_matches_the_oracle(ctx, n):
    arr = _random(n, 7 + n, 3, dead=0.4)
    g = _gpu(ctx, arr, n + 3, 3)
    o = _oracle(arr, n + 3, 3)
    st = Q.qp_compact_photons(ctx, g.handle)
    so = O.coalesce(o, None)
    assert st["n_after"] == so["n_after"] == int((arr["tau"] >= 0).sum()) == g.count()
    assert st["groups_merged"] == 0
    h = g.host()
    _compare(f"compact n={n}", h, o, 3, so["n_after"])
    # compaction moves data only: the state is the input's, in order
    alive = arr["tau"] >= 0
    np.testing.assert_array_equal(h["tau"], arr["tau"][alive])
    Q.qp_destroy_species(ctx, g.handle)


def test_arguments_are_checked(ctx):
    g = _gpu(ctx, _random(10, 1), 16, 3)
    el = DeviceSpecies(ctx, Q.QP_ELECTRON, 16, 3)
    bad = [Q.coalesce_params(PARAMS["box"], PARAMS["cells"], 3, 8, 3),   # not a power of 2
           Q.coalesce_params(PARAMS["box"], PARAMS["cells"], 8, 128, 3),
           Q.coalesce_params(PARAMS["box"], PARAMS["cells"], 8, 8, 2),
           Q.coalesce_params(PARAMS["box"], PARAMS["cells"], 8, 8, 5, max_group=4),
           Q.coalesce_params((0, 0, 0, 0.0, 1, 1), PARAMS["cells"], 8, 8, 3)]
    for p in bad:
        with pytest.raises(Q.QPError):
            Q.qp_coalesce_photons(ctx, g.handle, p)
    with pytest.raises(Q.QPError):  # leptons: a negative tau is not a sentinel
        Q.qp_compact_photons(ctx, el.handle)
    assert g.count() == 10


def test_cascade_with_periodic_coalescence_matches_the_oracle(ctx):
    # the constant-B cascade (FP64 path), coalesced every 10 steps; the
    # oracle restarts from the GPU state before each coalescence and takes
    # the same 10 steps and coalescence: renumbered photons keep drawing from
    # the streams of their new slots on both sides
    w = W.uniform_b_cascade(n=300, n_steps=60, cap=1 << 16)
    box = (-60.0, -60.0, -60.0, 7.5, 7.5, 7.5)
    sim = Simulation(w, precision="fp64", ctx=ctx)
    merged = 0
    for k in range(6):
        torch.cuda.synchronize()
        before = {nm: sp.host() for nm, sp in sim.species.items()}
        step = sim.step_index
        sim.run(10)
        p = Q.coalesce_params(box, (16, 16, 16), 4, 4, 3, seed=5, step=step + 10)
        st = Q.qp_coalesce_photons(ctx, sim.species["photon"].handle, p)
        merged += st["groups_merged"]
        torch.cuda.synchronize()
        _, osp = run_oracle_from_state(w, before, step, 10)
        so = O.coalesce(osp["photon"], O.coalesce_params(box, (16, 16, 16), 4, 4, 3, seed=5,
                                                         step=step + 10))
        g = sim.species["photon"].host()
        assert st["n_after"] == so["n_after"] and st["groups_merged"] == so["groups_merged"]
        o = oracle_arrays(osp["photon"])
        # the step leaves the two sides ~1e-15 apart; a merged pair's
        # transverse momentum sqrt((E/W)^2 - |P/W|^2) amplifies that for
        # nearly collinear groups, so momenta are compared against |u|
        assert momentum_error(g, o).max() <= 1e-12, k
        assert position_error(g, o).max() <= 1e-12, k
        np.testing.assert_allclose(g["w"], o["w"], rtol=1e-14, err_msg=f"round {k} w")
        for nm in ("electron", "positron"):
            ge, oe = sim.species[nm].host(), oracle_arrays(osp[nm])
            assert len(ge["x"]) == len(oe["x"])
            np.testing.assert_allclose(ge["ux"], oe["ux"], rtol=1e-12, atol=1e-9)
    assert merged > 0
    sim.close()


def test_coalesced_cascade_follows_the_kinetic_equations(ctx):
    # the paper's validation cascade (section 4) with the photons coalesced
    # every 50 steps: the weighted photon number and energy and the leptons
    # still follow Eq. 9-10 (the comparison without coalescence is in
    # test_gpu_cascade_kinetic.py)
    from oracle.kinetic import Cascade
    n = 1 << 16
    marks = (100, 200, 400)
    w = W.uniform_b_cascade(n=n, n_steps=400, cap=1 << 20)
    w["capacity"] = {"electron": n + (1 << 19), "positron": 1 << 19, "photon": 1 << 24}
    b0, dt = w["field"]["b0"], w["params"]["dt"]
    kin = Cascade(b0)
    p0 = math.sqrt(3000.0 ** 2 - 1.0)
    kms = [kin.moments(N) for N in kin.evolve(kin.initial_electrons(p0, 1.0),
                                              [m * dt for m in marks])]
    sim = Simulation(w, precision="mixed", ctx=ctx)
    box = (-80.0, -80.0, -80.0, 10.0, 10.0, 10.0)
    done, last = 0, None
    tol = {"n_electron": 0.04, "n_positron": 0.05, "n_photon": 0.04, "e_photon": 0.015,
           "e_electron": 0.06}
    for m, km in zip(marks, kms):
        while done < m:
            sim.run(50)
            done += 50
            last = Q.qp_coalesce_photons(ctx, sim.species["photon"].handle,
                                         Q.coalesce_params(box, (16, 16, 16), 8, 8, 3,
                                                           seed=9, step=done))
        torch.cuda.synchronize()
        d = {k: sim.diagnostics(k) for k in ("electron", "positron", "photon")}
        e_sub = d["electron"].e_subthreshold + d["positron"].e_subthreshold
        # weighted numbers: pairs from a merged photon carry its weight
        mc = {"n_electron": d["electron"].weight / n, "n_positron": d["positron"].weight / n,
              "n_photon": d["photon"].weight / n, "e_photon": (d["photon"].energy + e_sub) / n,
              "e_electron": d["electron"].energy / n}
        print(f"\n[coalesced step {m}] slots {d['photon'].n_live} (last merge {last}) "
              + " ".join(f"{k} {mc[k]:.4g}/{km[k]:.4g}" for k in mc))
        for k in mc:
            assert abs(mc[k] / km[k] - 1.0) <= tol[k], (m, k, mc[k], km[k])
        # coalescence holds the photon slots well below the weighted number
        assert d["photon"].n_live < 0.5 * d["photon"].weight
    sim.close()
