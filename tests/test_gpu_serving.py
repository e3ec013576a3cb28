"""Serving loop (continuous batching, CUDA graphs) on the GPU.

A request's results must not depend on what else is running: each request
served alone and in a mix with others (admitted while they run, different
sizes and step counts) ends in the same state, bit for bit, because every
launch computes each problem's tiles with the same arithmetic and appends in
the problem's own slot order.  The batched path also agrees with qp_step
(same kernels' arithmetic, per-problem descriptors in shared memory), graph
replays agree with direct launches, and admission respects device memory.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1311_1107_gb300 import qedpic as Q
from paper_1311_1107_gb300 import workloads as W
from paper_1311_1107_gb300.serve import ServingEngine
from paper_1311_1107_gb300.sim import Simulation

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = Q.qp_init_tables(W.LAMBDA_M, 0)
    yield c
    torch.cuda.synchronize()
    Q.qp_destroy(c)


REQS = [
    {"id": 0, "seed": 3, "n": 3000, "gamma": 2500.0, "a0": 300.0, "n_steps": 64, "arrival_s": 0.0},
    {"id": 1, "seed": 4, "n": 700, "gamma": 4000.0, "a0": 120.0, "n_steps": 40, "arrival_s": 0.0},
    {"id": 2, "seed": 5, "n": 5000, "gamma": 1500.0, "a0": 450.0, "n_steps": 88, "arrival_s": 0.002},
    {"id": 3, "seed": 6, "n": 1200, "gamma": 3000.0, "a0": 60.0, "n_steps": 24, "arrival_s": 0.004},
]


def serve(ctx, reqs, **kw):
    eng = ServingEngine(max_slots=kw.pop("max_slots", 8), arena_bytes=kw.pop("arena", 2 << 30),
                        graph_steps=kw.pop("graph_steps", 8), keep_state=True, ctx=ctx, **kw)
    try:
        out = eng.run(reqs)
    finally:
        eng.close()
    return out


def same_state(a, b):
    for sp in ("electron", "positron", "photon"):
        sa, sb = a[sp]["state"], b[sp]["state"]
        assert a[sp]["n_live"] == b[sp]["n_live"], sp
        for nm in sa:
            assert np.array_equal(sa[nm], sb[nm]), (sp, nm)


def test_results_same_alone_and_in_mix(ctx):
    alone = {r["id"]: serve(ctx, [dict(r, arrival_s=0.0)])["results"][0] for r in REQS}
    mix = serve(ctx, REQS)
    assert mix["max_concurrent"] >= 2
    for r in mix["results"]:
        same_state(r, alone[r["id"]])
        assert r["electron"]["n_emit"] == alone[r["id"]]["electron"]["n_emit"]
        assert r["photon"]["n_pair"] == alone[r["id"]]["photon"]["n_pair"]
        assert r["electron"]["status"] >= 0
    # every launch stepped every live slot of the request
    assert all(r["work"] >= r["n"] * r["n_steps"] for r in mix["results"])
    print(f"\n[serving mix] {len(mix['results'])} requests, max concurrent "
          f"{mix['max_concurrent']}, p50 {mix['p50_s'] * 1e3:.1f} ms, p99 "
          f"{mix['p99_s'] * 1e3:.1f} ms, {mix['throughput']:.3g} particle-steps/s")


def test_graph_replays_equal_direct_launches(ctx):
    a = serve(ctx, REQS[:2], use_graph=True)
    b = serve(ctx, REQS[:2], use_graph=False)
    for ra, rb in zip(a["results"], b["results"]):
        same_state(ra, rb)


def test_batched_request_matches_qp_step(ctx):
    r = REQS[0]
    res = serve(ctx, [r])["results"][0]
    w = W.serving_request_workload(r, 8)
    sim = Simulation(w, precision="mixed", ctx=ctx, track_chi=False)
    sim.run(r["n_steps"])
    torch.cuda.synchronize()
    for sp in ("electron", "positron", "photon"):
        h = sim.species[sp].host()
        st = res[sp]["state"]
        assert len(h["x"]) == len(st["x"]), sp
        for nm in st:
            if h.get(nm) is None:
                continue
            # same arithmetic; allow for a different contraction of a*b+c
            # by the compiler in the two instantiations
            err = np.abs(h[nm] - st[nm]) / np.maximum(np.abs(h[nm]), 1.0)
            assert err.max() <= 1e-9 if len(err) else True, (sp, nm, err.max())
    sim.close()


def test_admission_waits_for_device_memory(ctx):
    # three requests of one size and an arena that holds one at a time: all
    # complete, one after the other
    reqs = [dict(REQS[0], id=k, seed=10 + k, arrival_s=0.0) for k in range(3)]
    eng = ServingEngine(max_slots=8, arena_bytes=1 << 20, ctx=ctx)
    need = eng.bytes_for(reqs[0])
    eng.close()
    out = serve(ctx, reqs, arena=int(need * 1.5))
    assert len(out["results"]) == 3
    assert out["max_concurrent"] == 1
