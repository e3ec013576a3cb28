"""Multi-rank decomposition on CPU ranks (gloo, world size 2).

Each rank steps its slot range of one population with the oracle, its
particles keyed by their global ids; gathered, the primary particles (state
and per-particle event counts) equal a single-rank run of the whole
population bit for bit, and, with no pair creation, the emitted photons add
up to the same total.  The benchmark's reduction over ranks (slowest
time, total units) is checked on the same ranks.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1311_1107_gb300 import workloads as W  # noqa: E402
from paper_1311_1107_gb300.shard import (aggregate, shard_arrays, shard_ids,  # noqa: E402
                                          shard_range)

N, STEPS = 96, 40


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload():
    # no pairs: every emitter is a primary particle
    return W.plane_wave_collision(n=N, n_steps=STEPS)


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from tests.parity import oracle_arrays, run_oracle
        w = _workload()
        part, first = shard_arrays(w["electrons"], rank, world)
        ids = np.arange(first, first + len(part["x"]))
        # run_oracle with `sample` keeps each particle's global id
        osim, osp = run_oracle(w, STEPS, sample=ids)
        el = oracle_arrays(osp["electron"])
        local = {"first": first, "n": len(ids),
                 "el": {k: el[k][:len(ids)] for k in ("x", "y", "z", "ux", "uy", "uz", "tau",
                                                      "nemit")},
                 "photons": int(osp["photon"].n), "n_emit": int(osim.stats.n_emit)}
        gathered = [None] * world
        dist.all_gather_object(gathered, local)
        t, u = aggregate(10.0 + rank, 100 * (rank + 1), dist)
        if rank == 0:
            np.save(os.path.join(out_dir, "agg.npy"), np.array([t, u]))
            import pickle
            with open(os.path.join(out_dir, "parts.pkl"), "wb") as f:
                pickle.dump(gathered, f)
    finally:
        dist.destroy_process_group()


def test_shard_range_covers_in_order():
    for n in (0, 1, 7, 96, 131072):
        for world in (1, 2, 3, 8):
            parts = [shard_range(n, r, world) for r in range(world)]
            assert parts[0][0] == 0
            for (f0, c0), (f1, _) in zip(parts, parts[1:]):
                assert f0 + c0 == f1
            assert sum(c for _, c in parts) == n
            assert max(c for _, c in parts) - min(c for _, c in parts) <= 1


def test_two_ranks_reproduce_the_single_run(tmp_path):
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    import pickle
    parts = pickle.load(open(tmp_path / "parts.pkl", "rb"))
    t, u = np.load(tmp_path / "agg.npy")
    assert t == 11.0 and u == 300.0
    from tests.parity import oracle_arrays, run_oracle
    osim, osp = run_oracle(_workload(), STEPS)
    full = oracle_arrays(osp["electron"])
    for p in parts:
        a, b = p["first"], p["first"] + p["n"]
        for k, v in p["el"].items():
            assert np.array_equal(v, full[k][a:b]), k
    assert sum(p["n_emit"] for p in parts) == osim.stats.n_emit
    assert sum(p["photons"] for p in parts) == osp["photon"].n


def test_shard_ids_are_disjoint_and_keep_primaries():
    # every slot of every species of every rank gets a particle id no other
    # slot of that species uses; primary electrons keep their global ids;
    # one rank is the unsplit rule (slot i is particle i)
    cap = {"electron": 70, "positron": 40, "photon": 90}
    n_total = 61
    for world in (1, 2, 3, 5):
        seen = {k: set() for k in cap}
        for rank in range(world):
            first, count = shard_range(n_total, rank, world)
            rule = shard_ids(n_total, rank, world, cap)
            for sp, (base, split, app) in rule.items():
                for i in range(cap[sp]):
                    pid = app + (i - split) if split > 0 and i >= split else base + i
                    assert pid not in seen[sp], (world, rank, sp, i)
                    seen[sp].add(pid)
                    if sp == "electron" and i < count:
                        assert pid == first + i
            if world == 1:
                for sp, (base, split, app) in rule.items():
                    ids = [app + (i - split) if split > 0 and i >= split else base + i
                           for i in range(cap[sp])]
                    assert ids == list(range(cap[sp]))
