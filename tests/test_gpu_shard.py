"""The sharding key on the GPU: a population stepped as two parts, one after
the other, through shard.shard_arrays / shard.shard_ids and
Simulation(ids=...), against the oracle's run of the whole population and
against the whole population on the GPU (FP64 path; GPU only).

Every primary electron draws from the random streams of its global id, so
each part's primaries must equal the whole run's: slot by slot within 1e-6
of the oracle with identical per-particle event counts, and bit for bit
against the GPU's own unsplit run.  What a part appends gets ids no other
part uses, so its secondaries are statistically equivalent, not identical:
their totals are compared within Poisson noise."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1311_1107_gb300 import qedpic as Q
from paper_1311_1107_gb300 import workloads as W
from paper_1311_1107_gb300.shard import shard_arrays, shard_ids
from paper_1311_1107_gb300.sim import Simulation
from tests.parity import head, momentum_error, oracle_arrays, position_error, run_oracle

pytestmark = pytest.mark.gpu

KEYS = ("x", "y", "z", "ux", "uy", "uz", "tau")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = Q.qp_init_tables(W.LAMBDA_M, 0)
    yield c
    torch.cuda.synchronize()
    Q.qp_destroy(c)


def _part(w, rank, world):
    part, first = shard_arrays(w["electrons"], rank, world)
    wp = dict(w)
    wp["electrons"] = part
    return wp, first


def _run(ctx, w, n_steps, ids=None):
    sim = Simulation(w, precision="fp64", ctx=ctx, ids=ids)
    sim.run(n_steps)
    torch.cuda.synchronize()
    out = {n: sp.host() for n, sp in sim.species.items()}
    diag = {n: sim.diagnostics(n) for n in sim.species}
    return out, diag


CASES = {
    "plane wave, no pairs": (lambda: W.plane_wave_collision(n=601, n_steps=200), 200),
    "beam collision, pairs": (lambda: W.beam_collision(n=1001, n_steps=160, buffer=300_000), 160),
}


@pytest.mark.parametrize("case", list(CASES))
def test_two_parts_reproduce_the_whole_population(ctx, case):
    make, n_steps = CASES[case]
    w = make()
    n_all = len(w["electrons"]["x"])
    whole, whole_diag = _run(ctx, w, n_steps)
    osim, osp = run_oracle(w, n_steps)
    ora = oracle_arrays(osp["electron"])
    world = 2
    emitted = 0
    photons = 0
    for rank in range(world):
        wp, first = _part(w, rank, world)
        ids = shard_ids(n_all, rank, world, w["capacity"])
        n = len(wp["electrons"]["x"])
        assert ids["electron"][:2] == (first, n)
        got, diag = _run(ctx, wp, n_steps, ids)
        g = head(got["electron"], n)
        # bit for bit against the unsplit GPU run
        for k in KEYS + ("nemit",):
            np.testing.assert_array_equal(g[k], whole["electron"][k][first:first + n], k)
        # and against the oracle's whole population
        o = head(ora, n, np.arange(first, first + n))
        assert np.array_equal(g["nemit"], o["nemit"])
        eu, ex = momentum_error(g, o), position_error(g, o)
        print(f"\n[{case} part {rank}] {n} primaries: u max {eu.max():.3g}, x max {ex.max():.3g}, "
              f"events {int(g['nemit'].sum())}")
        assert eu.max() <= 1e-6 and ex.max() <= 1e-6
        emitted += int(diag["electron"].n_emit)
        photons += len(got["photon"]["x"])
    whole_emit = int(whole_diag["electron"].n_emit)
    whole_photons = len(whole["photon"]["x"])
    if not w["params"].get("pairs"):
        # every emitter is a primary: the totals are those of the whole run
        assert emitted == whole_emit and photons == whole_photons
    else:
        # pair products emit too, from other random streams: the same
        # physics, totals within Poisson noise
        assert abs(emitted - whole_emit) <= 5 * np.sqrt(whole_emit) + 5
        assert abs(photons - whole_photons) <= 5 * np.sqrt(whole_photons) + 5
