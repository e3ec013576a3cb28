"""qp_step launches captured in a CUDA graph (GPU only): a replay gives the
state that the same steps launched directly give, bit for bit.

The step kernel takes everything a launch needs from its parameters and
the device (live counts, tickets, look-back epoch), so a captured launch
replays the step it was captured with; the graph below holds two
consecutive steps, so the device-side reset of the tickets and the epoch
between launches is exercised inside the graph too."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1311_1107_gb300 import qedpic as Q
from paper_1311_1107_gb300 import workloads as W
from paper_1311_1107_gb300.sim import Simulation, stream_handle

pytestmark = pytest.mark.gpu

NAMES = ("electron", "positron", "photon")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = Q.qp_init_tables(W.LAMBDA_M, 0)
    yield c
    torch.cuda.synchronize()
    Q.qp_destroy(c)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_captured_steps_replay_like_direct_steps(ctx, precision):
    w = W.beam_collision(n=3000, n_steps=60, buffer=400_000)
    first = 35  # near the pulse peak: emissions and pairs in the captured steps
    ref = Simulation(w, precision=precision, ctx=ctx)
    ref.run(first + 2)
    torch.cuda.synchronize()

    sim = Simulation(w, precision=precision, ctx=ctx)
    sim.run(first)
    torch.cuda.synchronize()
    before = sim.live_counts()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    sim.params.n_steps = 1
    with torch.cuda.graph(g, stream=s):
        for k in (first, first + 1):
            sim.params.step = k
            Q.qp_step(sim.ctx, sim.params, stream_handle(s))
    torch.cuda.synchronize()
    # capturing runs nothing
    assert sim.live_counts() == before
    g.replay()
    torch.cuda.synchronize()
    got, want = sim.live_counts(), ref.live_counts()
    assert got == want
    assert want["photon"] > before["photon"] > 0
    for n in NAMES:
        a, b = sim.species[n].host(), ref.species[n].host()
        for f in b:
            assert np.array_equal(a[f], b[f], equal_nan=True), (n, f)
    for n in NAMES:
        da, db = sim.diagnostics(n), ref.diagnostics(n)
        assert da.status == db.status
        assert da.n_emit == db.n_emit and da.n_photon == db.n_photon and da.n_pair == db.n_pair
    del g
    sim.close()
    ref.close()
