"""Multi-GPU decomposition of the particle step (host logic only).

Given the fields, super-particles are independent, so the step shards with no
exchange: rank r owns a contiguous range of slots of one global population
and steps it on its own GPU.  Every particle's random streams are keyed by its
global id (species id_base + slot), so the primary particles of a sharded run
are bit-identical to a run of the whole population on one GPU; particles
appended during the run are numbered within their rank's buffers (their
draws, and so the secondaries, are statistically equivalent, not identical).
The only collective is the reduction of the benchmark's timing and counts.
"""
from __future__ import annotations


def shard_range(n_total: int, rank: int, world: int) -> tuple[int, int]:
    """(first, count) of rank's contiguous part of n_total slots; the parts
    differ in size by at most one and cover [0, n_total) in rank order."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n_total, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def shard_arrays(arrays: dict, rank: int, world: int) -> tuple[dict, int]:
    """The rank's slice of a population (dict of equal-length arrays) and the
    global id of its first particle."""
    n = len(next(iter(arrays.values())))
    first, count = shard_range(n, rank, world)
    return {k: v[first:first + count] for k, v in arrays.items()}, first


def shard_ids(n_total: int, rank: int, world: int, capacity: dict) -> dict:
    """Particle-id rule of each species of rank's part (species name ->
    (id_base, id_split, id_append) of qp_species_desc).  Primary electrons
    keep their global ids (first .. first + count - 1); what the rank appends
    gets ids no other rank uses: electrons from n_total + rank * cap_e on,
    positrons and photons from rank * cap on.  At world = 1 every slot i is
    particle i, as in an unsplit run.  capacity: slots per species on every
    rank (the same on all ranks)."""
    first, count = shard_range(n_total, rank, world)
    cap_e = int(capacity["electron"])
    if count > cap_e:
        raise ValueError("a rank's electrons exceed the electron capacity")
    return {
        "electron": (first, count, n_total + rank * cap_e) if count else
                    (n_total + rank * cap_e, 0, 0),
        "positron": (rank * int(capacity["positron"]), 0, 0),
        "photon": (rank * int(capacity["photon"]), 0, 0),
    }


def aggregate(time_ms: float, units: float, dist=None, device="cpu") -> tuple[float, float]:
    """Whole-job figures over ranks: the slowest rank's time and the total
    units processed (torch.distributed with any backend; identity at N=1)."""
    if dist is None:
        return float(time_ms), float(units)
    import torch
    t = torch.tensor([float(time_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())
