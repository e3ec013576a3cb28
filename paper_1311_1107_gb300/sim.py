"""Device-resident species and simulations on top of the C ABI.

PyTorch supplies the device memory (caller-owned buffers of the C ABI) and
streams; every step of the QED path runs in libqedpic's kernels.  A
``Simulation`` is built from a workload description of
``paper_1311_1107_gb300.workloads``.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import qedpic as Q
from .workloads import LAMBDA_M

NAMES = ("x", "y", "z", "ux", "uy", "uz", "tau", "w")
KIND = {"electron": Q.QP_ELECTRON, "positron": Q.QP_POSITRON, "photon": Q.QP_PHOTON}


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def stream_handle(stream) -> C.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class DeviceSpecies:
    """FP64 SoA buffers of one species on the GPU, registered with a context."""

    def __init__(self, ctx, kind: int, capacity: int, dims: int = 3, device="cuda:0",
                 track_chi: bool = True, id_base: int = 0, n_live=None, id_split: int = 0,
                 id_append: int = 0):
        """n_live: a one-element int64 device tensor to hold the live count
        (a view of a shared tensor lets a caller move all counts at once).
        id_base, id_split, id_append: the particle-id rule of the slots (the
        counters of their random streams, see qp_species_desc)."""
        self.kind, self.cap, self.dims = kind, int(capacity), dims
        n = max(self.cap, 1)
        names = [nm for nm in NAMES if not (nm == "z" and dims == 2)]
        # one allocation, array k at row k: the host copies of the state
        # (qp_species_copy) move every array of a species in one strided copy
        self.block = torch.zeros((len(names), n), dtype=torch.float64, device=device)
        self.t = {nm: self.block[k] for k, nm in enumerate(names)}
        self.chi = torch.zeros(n, dtype=torch.float64, device=device) if track_chi else None
        self.nemit = torch.zeros(n, dtype=torch.int32, device=device) if track_chi else None
        self.n_live = (n_live if n_live is not None
                       else torch.zeros(1, dtype=torch.int64, device=device))
        d = Q.qp_species_desc()
        d.kind, d.dims, d.capacity = kind, dims, self.cap
        for nm in NAMES:
            setattr(d, nm, _ptr(self.t.get(nm)))
        d.chi = _ptr(self.chi)
        d.nemit = _ptr(self.nemit)
        d.n_live = _ptr(self.n_live)
        d.id_base = int(id_base)
        d.id_split = int(id_split)
        d.id_append = int(id_append)
        self._desc = d
        self.ctx = ctx
        self.handle = Q.qp_create_species(ctx, d)

    def load(self, arrays: dict, n: int | None = None):
        """Copy initial particles into slots [0, n) and set the live count."""
        n = len(arrays["x"]) if n is None else n
        if n > self.cap:
            raise ValueError(f"{n} particles exceed capacity {self.cap}")
        if self.nemit is not None:
            self.nemit.zero_()
        for nm, t in self.t.items():
            if nm in arrays and n:
                t[:n].copy_(torch.as_tensor(np.asarray(arrays[nm][:n], dtype=np.float64)))
        self.n_live.fill_(n)

    def copy_state(self, host: torch.Tensor, count: int, to_device: bool, stream=None):
        """Slots [0, count) of the FP64 arrays between the device and a host
        tensor shaped like self.block (pinned for asynchronous copies)."""
        Q.qp_species_copy(self.ctx, self.handle, host.data_ptr(), host.stride(0) * 8, count,
                          to_device, stream)

    def count(self) -> int:
        return int(self.n_live.item())

    def host(self, n: int | None = None) -> dict:
        n = self.count() if n is None else n
        out = {nm: t[:n].cpu().numpy() for nm, t in self.t.items()}
        if self.chi is not None:
            out["chi"] = self.chi[:n].cpu().numpy()
        if self.nemit is not None:
            out["nemit"] = self.nemit[:n].cpu().numpy()
        return out


def make_field(desc: dict, device="cuda:0"):
    """qp_field from a workload field description (Yee components are
    uploaded to device float32 arrays that the field keeps alive)."""
    f = Q.qp_field()
    f.kind = Q.FIELD_KINDS[desc["kind"]]
    f.a0 = desc.get("a0", 0.0)
    f.w0 = desc.get("w0", 0.0)
    f.tau_fwhm = desc.get("tau_fwhm", 0.0)
    f.x_focus = desc.get("x_focus", 0.0)
    f.t_focus = desc.get("t_focus", 0.0)
    f.b0 = desc.get("b0", 0.0)
    keep = []
    if desc["kind"] == "yee2d":
        comps = [torch.as_tensor(np.ascontiguousarray(c, dtype=np.float32)).to(device)
                 for c in desc["comps"]]
        keep = comps
        for k, c in enumerate(comps):
            f.yee[k] = c.data_ptr()
        f.ny, f.nx = comps[0].shape
        f.dx, f.dy = desc["dx"], desc["dy"]
        f.x0, f.y0 = desc.get("x0", 0.0), desc.get("y0", 0.0)
    return f, keep


class Simulation:
    """One run: a context, three species and the step parameters."""

    def __init__(self, workload: dict, precision: str = "fp64", device: int = 0, ctx=None,
                 track_chi: bool = True, init_tau: bool = True, load: bool = True,
                 id_base: int = 0, ids: dict | None = None):
        """id_base: particle id of the first electron slot (a shard of a larger
        population keeps its particles' random streams).  ids: optional
        species name -> (id_base, id_split, id_append), the id rule of each
        species (shard.shard_ids); it replaces id_base."""
        self.dev = f"cuda:{device}"
        self.own_ctx = ctx is None
        self.ctx = ctx if ctx is not None else Q.qp_init_tables(LAMBDA_M, device)
        self.workload = workload
        dims = workload["dims"]
        cap = workload["capacity"]
        # live counts of electrons, positrons, photons side by side
        self.counts = torch.zeros(3, dtype=torch.int64, device=self.dev)
        if ids is None:
            ids = {"electron": (id_base, 0, 0), "positron": (0, 0, 0), "photon": (0, 0, 0)}
        self.species = {
            name: DeviceSpecies(self.ctx, KIND[name], cap[name], dims, self.dev, track_chi,
                                ids[name][0], n_live=self.counts[k:k + 1],
                                id_split=ids[name][1], id_append=ids[name][2])
            for k, name in enumerate(("electron", "positron", "photon"))
        }
        self.field, self._keep = make_field(workload["field"], self.dev)
        rf = workload["field"].get("refill")
        self.pulse = (Q.pulse2d(rf["a0"], rf["w0"], rf["tau_fwhm"], rf["x_focus"],
                                rf["t_focus"], rf["y_axis"]) if rf else None)
        pc = workload["field"].get("pic")
        self.pic_pulse = (Q.pulse2d(pc["a0"], pc["w0"], pc["tau_fwhm"], pc["x_focus"],
                                    pc["t_focus"], pc["y_axis"]) if pc else None)
        self.J = None
        if pc:
            ny, nx = workload["field"]["comps"][0].shape
            self.J = torch.zeros((3, ny, nx), dtype=torch.float32, device=self.dev)
        p = workload["params"]
        s = Q.qp_step_params()
        s.field = self.field
        s.dt = p["dt"]
        s.precision = Q.QP_MIXED if precision == "mixed" else Q.QP_FP64
        s.seed = int(p.get("seed", 0))
        s.chi_threshold = float(p.get("chi_th", 0.0))
        s.photon_min_gamma = float(p.get("photon_min_gamma", 2.0))
        s.pairs = 1 if p.get("pairs", False) else 0
        s.max_emissions = int(p.get("max_emit", 8))
        s.electron = self.species["electron"].handle
        s.positron = self.species["positron"].handle
        s.photon = self.species["photon"].handle
        self.params = s
        self.step_index = int(p.get("step", 0))
        if load:
            self.load_initial(init_tau)

    def load_initial(self, init_tau: bool = True, stream=None):
        if self.pic_pulse is not None:
            # the grid starts with the pulse at the first step's time (E and
            # B at that time); the solver advances it from there
            for c in self._keep:
                c.zero_()
            t0 = int(self.workload["params"].get("step", 0)) * self.workload["params"]["dt"]
            Q.qp_fill_yee2d(self.ctx, self.pic_pulse, self.field, t0, stream_handle(stream))
        el = self.species["electron"]
        el.load(self.workload["electrons"])
        for sp in ("positron", "photon"):
            self.species[sp].n_live.zero_()
        if init_tau:
            n = len(self.workload["electrons"]["x"])
            Q.qp_init_optical_depth(self.ctx, el.handle, self.params.seed, 0, n,
                                    stream_handle(stream))
        for sp in self.species.values():
            Q.qp_reset_counters(self.ctx, sp.handle)
        self.step_index = int(self.workload["params"].get("step", 0))

    def run_fused(self, n_steps: int, fuse: int, stream=None) -> int:
        """n_steps steps in launch windows of `fuse` steps (qp_step_fused:
        pairs off, fixed or analytic fields)."""
        self.params.step = self.step_index
        self.params.n_steps = int(n_steps)
        st = Q.qp_step_fused(self.ctx, self.params, int(fuse), stream_handle(stream))
        self.step_index += int(n_steps)
        return st

    def _pic_step(self, sh) -> int:
        """One PIC cycle: B half step, the QED step, the current, B half
        step, E full step (E^n and B^(n-1/2) stored between cycles)."""
        dt = self.params.dt
        Q.qp_yee_advance_b(self.ctx, self.field, 0.5 * dt, sh)
        self.params.step = self.step_index
        self.params.n_steps = 1
        st = Q.qp_step(self.ctx, self.params, sh)
        self.J.zero_()
        j = [self.J[k].data_ptr() for k in range(3)]
        for name in ("electron", "positron"):
            sp = self.species[name]
            if sp.cap > 0:
                Q.qp_deposit_current(self.ctx, sp.handle, self.field, j[0], j[1], j[2], dt, sh)
        Q.qp_yee_advance_b(self.ctx, self.field, 0.5 * dt, sh)
        Q.qp_yee_advance_e(self.ctx, self.field, j[0], j[1], j[2], dt, sh)
        self.step_index += 1
        return st

    def run(self, n_steps: int, stream=None) -> int:
        if self.pic_pulse is not None:
            sh = stream_handle(stream)
            st = 0
            for _ in range(int(n_steps)):
                st = max(st, self._pic_step(sh))
            return st
        if self.pulse is not None:
            # fields refilled from the pulse at each step's time, then the step
            st = 0
            for _ in range(int(n_steps)):
                Q.qp_fill_yee2d(self.ctx, self.pulse, self.field,
                                self.step_index * self.params.dt, stream_handle(stream))
                self.params.step = self.step_index
                self.params.n_steps = 1
                st = max(st, Q.qp_step(self.ctx, self.params, stream_handle(stream)))
                self.step_index += 1
            return st
        self.params.step = self.step_index
        self.params.n_steps = int(n_steps)
        st = Q.qp_step(self.ctx, self.params, stream_handle(stream))
        self.step_index += int(n_steps)
        return st

    def host_states(self, host: dict, counts: dict):
        """qp_host_state[3] over host blocks shaped like the species' blocks
        (pinned tensors, array k in row k) holding counts[name] live slots."""
        arr = (Q.qp_host_state * 3)()
        for k, name in enumerate(("electron", "positron", "photon")):
            h = host[name]
            arr[k].host = h.data_ptr()
            arr[k].pitch = h.stride(0) * h.element_size()
            arr[k].count = int(counts[name])
        return arr

    def run_host(self, states, n_steps: int = 1, stream=None) -> int:
        """n_steps steps of state held in host blocks (qp_step_host): copied
        in, stepped, copied back; states[k].count become the new counts."""
        if self.pulse is not None or self.pic_pulse is not None:
            raise ValueError("run_host steps a workload with given fields only")
        self.params.step = self.step_index
        self.params.n_steps = int(n_steps)
        st = Q.qp_step_host(self.ctx, self.params, states, stream_handle(stream))
        self.step_index += int(n_steps)
        return st

    def diagnostics(self, name: str, stream=None) -> Q.qp_diag:
        return Q.qp_diagnostics(self.ctx, self.species[name].handle, stream_handle(stream))

    def live_counts(self) -> dict:
        return {k: v.count() for k, v in self.species.items()}

    def close(self):
        if self.own_ctx and self.ctx is not None:
            torch.cuda.synchronize()
            Q.qp_destroy(self.ctx)
            self.ctx = None
