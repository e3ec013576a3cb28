"""Serving loop: continuous batching of independent beam-laser collision runs.

Requests (beam collisions of different particle counts, energies, pulse
amplitudes, step counts and seeds) arrive over time.  Each is admitted as soon
as a batch slot and enough device memory are free: its particle, photon and
pair buffers are carved from one resident device arena, its electrons are
copied in and its optical depths drawn, and it becomes one problem of a
libqedpic batch.  The GPU runs CUDA-graph replays of K shared launches
(qp_batch_step): every launch takes one step of every active request, so
requests of any size overlap on the device.  A request leaves when its steps
are done (its step counter lives on the device); its results are the species
diagnostics (and, optionally, its final state), read on a side stream while
the others keep running.  The engine records each request's latency (arrival
to results), and the throughput in particle-steps.

Every step of every request runs in libqedpic's kernels; this module only
allocates, copies and schedules.
"""
from __future__ import annotations

import ctypes as C
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import qedpic as Q
from .sim import NAMES, stream_handle
from .workloads import LAMBDA_M, serving_request_workload

ALIGN = 256
KINDS = (("electron", Q.QP_ELECTRON), ("positron", Q.QP_POSITRON), ("photon", Q.QP_PHOTON))


class Arena:
    """First-fit allocator over one resident device buffer (256-byte blocks)."""

    def __init__(self, nbytes: int, device: str):
        self.size = int(nbytes) // ALIGN * ALIGN
        self.buf = torch.empty(self.size, dtype=torch.uint8, device=device)
        self.base = self.buf.data_ptr()
        self.free = [(0, self.size)]  # sorted, disjoint (offset, size)
        self.used = 0

    @staticmethod
    def rounded(nbytes: int) -> int:
        return (int(nbytes) + ALIGN - 1) // ALIGN * ALIGN

    def alloc(self, nbytes: int):
        n = self.rounded(nbytes)
        for k, (off, size) in enumerate(self.free):
            if size >= n:
                if size == n:
                    self.free.pop(k)
                else:
                    self.free[k] = (off + n, size - n)
                self.used += n
                return off
        return None

    def release(self, off: int, nbytes: int):
        n = self.rounded(nbytes)
        self.used -= n
        self.free.append((off, n))
        self.free.sort()
        merged = []
        for o, s in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + s)
            else:
                merged.append((o, s))
        self.free = merged

    def view(self, off: int, count: int, dtype) -> torch.Tensor:
        item = torch.empty(0, dtype=dtype).element_size()
        return self.buf[off:off + count * item].view(dtype)


def _tiles(n: int) -> int:
    return (n + Q.QP_STEP_TILE - 1) // Q.QP_STEP_TILE


@dataclass
class Admitted:
    req: dict
    slot: int
    off: int
    nbytes: int
    handles: dict
    tensors: dict
    caps: dict
    replay_set: int          # first replay index whose progress includes this slot
    t_admit: float
    staged: list = field(default_factory=list)


class ServingEngine:
    """One GPU, one context, one batch of `max_slots` problems, one arena."""

    def __init__(self, max_slots: int = 32, arena_bytes: int = 16 << 30, graph_steps: int = 8,
                 capacity_factor: int = 8, device: int = 0, use_graph: bool = True,
                 keep_state: bool = False, ctx=None):
        self.dev = f"cuda:{device}"
        self.device = device
        self.own_ctx = ctx is None
        self.ctx = ctx if ctx is not None else Q.qp_init_tables(LAMBDA_M, device)
        self.max_slots = int(max_slots)
        self.batch = Q.qp_batch_create(self.ctx, self.max_slots, Q.QP_MIXED, Q.QP_FIELD_GAUSSIAN)
        self.K = int(graph_steps)
        self.cf = int(capacity_factor)
        self.keep_state = keep_state
        self.stream = torch.cuda.Stream(device=self.dev)
        self.side = torch.cuda.Stream(device=self.dev)
        self.arena = Arena(arena_bytes, self.dev)
        self.free_slots = list(range(self.max_slots))
        self.active: dict[int, Admitted] = {}
        self.left = [torch.zeros(self.max_slots, dtype=torch.int64).pin_memory() for _ in range(2)]
        self.work = [torch.zeros(self.max_slots, dtype=torch.int64).pin_memory() for _ in range(2)]
        self.events = [torch.cuda.Event() for _ in range(2)]
        self.replays = 0
        self.graph = None
        if use_graph:
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph, stream=self.stream):
                Q.qp_batch_step(self.batch, self.K, stream_handle(self.stream))
        self.max_concurrent = 0

    # ------------------------------------------------------------ memory
    def species_caps(self, req: dict) -> dict:
        n = int(req["n"])
        buf = self.cf * n
        return {"electron": n + buf, "positron": buf, "photon": buf}

    def bytes_for(self, req: dict) -> int:
        caps = self.species_caps(req)
        b = 0
        for name, _ in KINDS:
            b += len(NAMES) * Arena.rounded(8 * max(caps[name], 1)) + ALIGN  # arrays + n_live
        words = _tiles(caps["electron"]) + _tiles(caps["positron"]) + _tiles(caps["photon"]) + 8
        return b + Arena.rounded(8 * words)

    # ------------------------------------------------------------ admission
    def try_admit(self, req: dict, payload: dict | None = None) -> bool:
        if not self.free_slots:
            return False
        need = self.bytes_for(req)
        off = self.arena.alloc(need)
        if off is None:
            return False
        slot = self.free_slots.pop(0)
        caps = self.species_caps(req)
        w = payload if payload is not None else serving_request_workload(req, self.cf)
        cur = off
        tensors, handles = {}, {}
        for name, kind in KINDS:
            cap = caps[name]
            t = {}
            for nm in NAMES:
                t[nm] = self.arena.view(cur, cap, torch.float64)
                cur += Arena.rounded(8 * max(cap, 1))
            t["n_live"] = self.arena.view(cur, 1, torch.int64)
            cur += ALIGN
            d = Q.qp_species_desc()
            d.kind, d.dims, d.capacity = kind, 3, cap
            for nm in NAMES:
                setattr(d, nm, C.c_void_p(t[nm].data_ptr()))
            d.chi = None
            d.nemit = None
            d.n_live = C.c_void_p(t["n_live"].data_ptr())
            handles[name] = Q.qp_create_species(self.ctx, d)
            tensors[name] = t
        scratch_off = cur
        s = self._params(w, handles, int(req["n_steps"]))
        words = Q.qp_batch_scratch_words(self.ctx, s)
        assert scratch_off + 8 * words <= off + Arena.rounded(need)
        el = w["electrons"]
        n = len(el["x"])
        staged = []  # pinned copies of the payload, alive until the request leaves
        with torch.cuda.stream(self.stream):
            te = tensors["electron"]
            for nm in NAMES:
                if nm in el and n:
                    src = torch.from_numpy(np.ascontiguousarray(el[nm], dtype=np.float64))
                    src = src.pin_memory()
                    staged.append(src)
                    te[nm][:n].copy_(src, non_blocking=True)
            te["n_live"].fill_(n)
            tensors["positron"]["n_live"].zero_()
            tensors["photon"]["n_live"].zero_()
        st = stream_handle(self.stream)
        Q.qp_init_optical_depth(self.ctx, handles["electron"], int(w["params"]["seed"]), 0, n, st)
        Q.qp_batch_set(self.batch, slot, s, self.arena.base + scratch_off, words, st)
        self.active[slot] = Admitted(req, slot, off, need, handles, tensors, caps,
                                     self.replays, time.perf_counter(), staged)
        self.max_concurrent = max(self.max_concurrent, len(self.active))
        return True

    def _params(self, w: dict, handles: dict, n_steps: int) -> Q.qp_step_params:
        f = Q.qp_field()
        fd = w["field"]
        f.kind = Q.QP_FIELD_GAUSSIAN
        f.a0, f.w0, f.tau_fwhm = fd["a0"], fd["w0"], fd["tau_fwhm"]
        f.x_focus, f.t_focus = fd["x_focus"], fd["t_focus"]
        p = w["params"]
        s = Q.qp_step_params()
        s.field = f
        s.dt = p["dt"]
        s.step = 0
        s.n_steps = n_steps
        s.precision = Q.QP_MIXED
        s.seed = int(p["seed"])
        s.chi_threshold = float(p["chi_th"])
        s.photon_min_gamma = float(p["photon_min_gamma"])
        s.pairs = 1 if p["pairs"] else 0
        s.max_emissions = int(p["max_emit"])
        s.electron = handles["electron"]
        s.positron = handles["positron"]
        s.photon = handles["photon"]
        return s

    # ------------------------------------------------------------ stepping
    def replay(self):
        """K shared launches, then an asynchronous copy of the progress."""
        k = self.replays % 2
        with torch.cuda.stream(self.stream):
            if self.graph is not None:
                self.graph.replay()
            else:
                Q.qp_batch_step(self.batch, self.K, stream_handle(self.stream))
            Q.qp_batch_progress(self.batch, self.left[k].data_ptr(), None,
                                self.work[k].data_ptr(), stream_handle(self.stream))
            self.events[k].record(self.stream)
        self.replays += 1

    def retire_finished(self, replay_index: int, t0: float) -> list:
        """Requests found finished in the progress of replay `replay_index`
        (already completed on the device): results read, memory freed."""
        k = replay_index % 2
        self.events[k].synchronize()
        left = self.left[k].numpy()
        work = self.work[k].numpy()
        done = []
        for slot, a in list(self.active.items()):
            if replay_index < a.replay_set or left[slot] > 0:
                continue
            self.side.wait_event(self.events[k])
            res = {"id": a.req["id"], "work": int(work[slot]),
                   "n_steps": int(a.req["n_steps"]), "n": int(a.req["n"])}
            sh = stream_handle(self.side)
            for name, _ in KINDS:
                d = Q.qp_diagnostics(self.ctx, a.handles[name], sh)
                res[name] = {"n_live": d.n_live, "n_alive": d.n_alive, "energy": d.energy,
                             "weight": d.weight, "n_emit": d.n_emit, "n_pair": d.n_pair,
                             "n_photon": d.n_photon, "n_dropped": d.n_photon_drop + d.n_pair_drop,
                             "status": d.status}
                if self.keep_state:
                    with torch.cuda.stream(self.side):
                        n = d.n_live
                        res[name]["state"] = {nm: a.tensors[name][nm][:n].cpu().numpy()
                                              for nm in NAMES}
            self.side.synchronize()
            t = time.perf_counter()
            res["latency_s"] = t - t0 - a.req["arrival_s"]
            res["queue_s"] = a.t_admit - t0 - a.req["arrival_s"]
            for name, _ in KINDS:
                Q.qp_destroy_species(self.ctx, a.handles[name])
            self.arena.release(a.off, a.nbytes)
            self.free_slots.append(slot)
            self.free_slots.sort()
            del self.active[slot]
            done.append(res)
        return done

    def run(self, requests: list, payloads: dict | None = None, time_scale: float = 1.0) -> dict:
        """Serve `requests` (dicts with id, n, gamma, a0, n_steps, seed,
        arrival_s) in arrival order; arrival times are multiplied by
        time_scale.  Returns per-request results and aggregate figures."""
        reqs = sorted(({**r, "arrival_s": r["arrival_s"] * time_scale} for r in requests),
                      key=lambda r: r["arrival_s"])
        pending = list(reqs)
        results = []
        torch.cuda.synchronize(self.dev)
        t0 = time.perf_counter()
        last_checked = -1
        while pending or self.active:
            now = time.perf_counter() - t0
            while pending and pending[0]["arrival_s"] <= now:
                r = pending[0]
                if not self.try_admit(r, None if payloads is None else payloads.get(r["id"])):
                    break
                pending.pop(0)
            if not self.active:
                if pending:
                    time.sleep(max(0.0, min(pending[0]["arrival_s"] - now, 0.01)))
                continue
            self.replay()
            # results of the previous replay, while this one runs
            if self.replays >= 2:
                last_checked = self.replays - 2
                results += self.retire_finished(last_checked, t0)
        # the last replay's progress
        if self.replays - 1 > last_checked:
            results += self.retire_finished(self.replays - 1, t0)
        torch.cuda.synchronize(self.dev)
        makespan = time.perf_counter() - t0
        lat = np.array([r["latency_s"] for r in results]) if results else np.zeros(1)
        work = sum(r["work"] for r in results)
        return {"results": sorted(results, key=lambda r: r["id"]), "makespan_s": makespan,
                "particle_steps": work, "throughput": work / makespan if makespan > 0 else 0.0,
                "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "max_concurrent": self.max_concurrent, "replays": self.replays}

    def close(self):
        torch.cuda.synchronize(self.dev)
        if self.batch is not None:
            Q.qp_batch_destroy(self.batch)
            self.batch = None
        self.graph = None
        if self.own_ctx and self.ctx is not None:
            Q.qp_destroy(self.ctx)
            self.ctx = None
