#!/usr/bin/env python
"""Benchmark of the QED particle step on GB300.

Default workload: the 2D laser-on-foil case (2048x512 Yee grid, 131072 e-,
fixed Gaussian-pulse fields, Sokolov below chi 1e-3, Monte-Carlo above,
photons and pairs tracked), run on the mixed-precision path (the headline
`value`) and on the FP64 path (`fp64`) on the same GPU.  A step is one
qp_step (one launch of the fused step kernel) over every live particle;
K steps are timed from the initial state (K = 500 is the whole job).
The line also carries
  `collision`: the beam collision at full size (1e7 e-, 1e8-slot photon
      and pair buffers, the K steps from step 980, around the pulse peak),
      mixed and FP64, each with its roofline: the many-particle state in
      which the step's HBM bound can be approached;
  `pic`: the same foil as a PIC cycle (Yee solver and current deposition
      around every QED step: qp_yee_advance_*, qp_deposit_current);
  `fused`: the plane-wave case (4096 e-, 1000 steps, no pairs) as one job,
      one launch a step against one fused window of 1000 steps, FP64 and
      mixed;
  `refill`: the same foil with its E_y and B_z refilled from the pulse
      before every step (qp_fill_yee2d), mixed and FP64;
  `serving`: the 256-request stream of beam-collision requests (n_e
      log-uniform 1e3-1e6) served with continuous batching (Poisson arrivals
      at ~70 % of the measured batched throughput), its throughput and
      p50/p99 request latency;
  `e2e`: the same steps through the public API with the state copied from
      and to pinned host memory every step;
  `cpu_baseline`: the FP64 oracle on a bounded sample, on one core and on
      every host core.
Particle-steps count the live slots at each step start, decayed photons
(tau < 0, kept in their slots) left out.  L2 is flushed (256 MB write)
between timed steps; each step is timed with CUDA events on its stream,
queued by the host ahead of the device (~1 ms of flushes before the first
timed step); clocks are sampled with nvidia-smi meanwhile.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload foil|collision|plane|serving] [--requests R]

Under torchrun each rank steps its own shard of a population of N copies of
the workload (disjoint particle ids, so every particle has its own random
streams) on its own GPU: weak scaling with no collective in the data path;
the barrier and the max over ranks of the timed region come from
torch.distributed.  The reference arm (`--impl reference`) is the CPU
oracle on every host core: the paper has no code to install.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "QED particle-steps/s, mixed vs FP64 on same GPU; p50/p99 request latency"
UNIT = "particle-steps/s"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
PROFILES = os.path.join(ROOT, "profiles")
FALLBACK_HBM_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=500)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=("ours", "reference"), default="ours")
    p.add_argument("--workload", choices=("foil", "collision", "plane", "serving", "fused",
                                          "coalesce", "refill", "pic"),
                   default="foil")
    p.add_argument("--requests", type=int, default=None,
                   help="serving: requests in the stream (default 256)")
    p.add_argument("--serving-nmax", type=float, default=None,
                   help="serving: largest electron count of a request (default 1e6)")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--no-collision", action="store_true",
                   help="leave the full-size collision leg out of the default line")
    p.add_argument("--collision-n", type=float, default=None,
                   help="collision: electrons (default 1e7; buffers 10x)")
    p.add_argument("--start-step", type=int, default=None,
                   help="collision: first step of the timed window (the beam is placed where "
                        "it is then; default 980, the steps around the pulse peak)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--e2e-steps", type=int, default=100)
    p.add_argument("--ref-cores", type=int, default=None,
                   help="reference arm: host cores (processes) to time the oracle on "
                        "(default: every core of the host)")
    return p.parse_args()


def workload(name: str, seed: int, start_step: int | None = None, collision_n=None):
    from paper_1311_1107_gb300 import workloads as W
    if name == "foil":
        return W.laser_on_foil(seed=seed)
    if name == "refill":  # the foil, its fields refilled from the pulse before every step
        return W.laser_on_foil(seed=seed, refill=True)
    if name == "pic":  # the foil as a PIC cycle (Yee solver and current around each step)
        return W.laser_on_foil(seed=seed, pic=True)
    if name == "collision":
        # the 1e7-electron collision, timed from `start` (default 980: the
        # window around the pulse peak at step 1000), the beam placed where
        # it is then (it moves at ~c along -x before meeting the pulse)
        n = int(collision_n or 10_000_000)
        w = W.beam_collision(n=n, buffer=10 * n, seed=seed)
        start = 980 if start_step is None else start_step
        w["electrons"]["x"] = w["electrons"]["x"] - start * w["params"]["dt"]
        w["params"]["step"] = start
        w["name"] += f", timed from step {start}"
        return w
    if name == "serving":
        return W.serving_request_workload(W.serving_requests(n_requests=1, seed=seed)[0])
    return W.plane_wave_collision(seed=seed)


# ----------------------------------------------------------------------------- bytes model

def species_bytes(dims: int, pairs: bool):
    """Algorithmic HBM bytes: per lepton slot-step (x, u, tau read and
    written), per photon slot-step (x, u, tau read; x and, with pairs, tau
    written), per appended particle (its 7-8 arrays) and per emitting parent
    (its weight)."""
    pos = 8 * dims
    lep = 2 * (pos + 24 + 8)
    pho = pos + 24 + 8 + pos + (8 if pairs else 0)
    new = pos + 24 + 8 + 8
    return lep, pho, new


DEAD_B = 8  # a decayed photon's slot: its optical-depth sentinel is read


def peaks():
    try:
        with open(PEAKS) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons (200 ms)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [s.strip() for s in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ----------------------------------------------------------------------------- GPU path

def run_path(w, precision, steps, warmup, dev, dist, flush, ids=None):
    import torch

    from paper_1311_1107_gb300 import qedpic as Q
    from paper_1311_1107_gb300.sim import Simulation
    from paper_1311_1107_gb300.workloads import LAMBDA_M

    ctx = Q.qp_init_tables(LAMBDA_M, dev)
    sim = Simulation(w, precision=precision, ctx=ctx, device=dev, track_chi=False, ids=ids)
    stream = torch.cuda.current_stream()
    names = ("electron", "positron", "photon")
    counts = torch.zeros((steps, 3), dtype=torch.int64, device=f"cuda:{dev}")
    live = [sim.species[n].n_live for n in names]
    # warm-up steps on the initial state (the timed loop's own launches, so
    # that every kernel and event the loop uses has run once), then back to
    # the initial state
    for _ in range(warmup):
        flush.zero_()
        torch.cat(live, out=counts[0])
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.run(1)
        b.record(stream)
    torch.cuda.synchronize()
    sim.load_initial()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    # A step of a workload with given fields is one k_step launch: its own
    # events time the kernel.  Where a step also refills or advances the
    # grid, the library's per-launch events time k_step among the step's
    # launches (they add ~4 us of event records to each such step).
    single = sim.pulse is None and sim.pic_pulse is None
    Q.qp_profile_enable(ctx, not single)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    # ~1 ms of L2 flushes ahead of the first timed step: the host queues the
    # steps before the device reaches them (and stays ahead: a step's flush
    # alone outlasts the host's loop), so the events time the device's work
    # and not the Python loop between launches; real work, not an idle
    # spin, so the clocks stay up
    for _ in range(25):
        flush.zero_()
    for k in range(steps):
        flush.zero_()
        torch.cat(live, out=counts[k])       # live slots at the start of the step
        ev[k][0].record(stream)
        sim.run(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if dist:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    if single:
        ms, launches = [sum(step_ms), 0.0, 0.0], [steps, 0, 0]
    else:
        ms, launches = Q.qp_profile_read(ctx)
    Q.qp_profile_enable(ctx, False)
    c = counts.cpu().numpy()
    diag = {n: sim.diagnostics(n) for n in names}
    lep_slots = int(c[:, 0].sum() + c[:, 1].sum())
    # photons that decayed keep their slot (tau < 0) and are only tested:
    # each pair event kills one photon and appends one electron, so the dead
    # slots at the start of step k are the electrons appended since step 0
    # (exact while no pair was dropped at the capacity)
    dead = c[:, 0] - c[0, 0]
    pho_all = int(c[:, 2].sum())
    pho_slots = int((c[:, 2] - dead).sum())
    res = {
        "ctx": ctx, "sim": sim, "step_ms": step_ms, "kernel_ms": ms, "launches": launches,
        "lep_slots": lep_slots, "pho_slots": pho_slots, "dead_slots": pho_all - pho_slots,
        "pair_drops": int(diag["photon"].n_pair_drop), "wall_s": wall,
        "photons_added": int(sum(diag[n].n_photon for n in ("electron", "positron"))),
        "pairs_added": int(diag["photon"].n_pair - diag["photon"].n_pair_drop),
        "emitters": int(sum(diag[n].n_emit for n in ("electron", "positron"))),
        "final_live": {n: int(sim.species[n].count()) for n in names},
        "status": min(d.status for d in diag.values()),
    }
    return res


def fused_leg(dev, flush, warmup: int):
    """The plane-wave case (4096 e-, 1000 steps, no pairs) run as one job:
    one launch a step (qp_step) against fused windows (qp_step_fused, the
    whole job in one window of 1000 steps), FP64 and mixed.  L2 is flushed
    before each timed job; the particle-steps are the live slots at each
    step start (an untimed single-step run counts them; the fused run has
    the same slots, bit for bit)."""
    import torch

    from paper_1311_1107_gb300 import qedpic as Q
    from paper_1311_1107_gb300 import workloads as W
    from paper_1311_1107_gb300.sim import Simulation

    w = W.plane_wave_collision()
    n_steps = int(w["params"]["n_steps"])
    ctx = Q.qp_init_tables(W.LAMBDA_M, dev)
    out = {"workload": w["name"], "fuse": n_steps}
    stream = torch.cuda.current_stream()
    for prec in ("fp64", "mixed"):
        sim = Simulation(w, precision=prec, ctx=ctx, device=dev, track_chi=False)
        names = ("electron", "positron", "photon")
        counts = torch.zeros((n_steps, 3), dtype=torch.int64, device=f"cuda:{dev}")
        live = [sim.species[n].n_live for n in names]
        for k in range(n_steps):
            torch.cat(live, out=counts[k])
            sim.run(1)
        slots = int(counts.sum().item())

        def job(fused):
            sim.load_initial()
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            if fused:
                sim.run_fused(n_steps, n_steps)
            else:
                sim.run(n_steps)
            b.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b)

        for _ in range(max(1, warmup)):
            job(False)
            job(True)
        t1 = job(False)
        Q.qp_profile_enable(ctx, True)
        tf = job(True)
        win_ms, wins = Q.qp_profile_read(ctx)
        Q.qp_profile_enable(ctx, False)
        out[prec] = {"single_steps": {"value": round(slots / (t1 * 1e-3), 1), "unit": UNIT,
                                      "ms_per_step": round(t1 / n_steps, 5)},
                     "fused": {"value": round(slots / (tf * 1e-3), 1), "unit": UNIT,
                               "ms_per_step": round(tf / n_steps, 5)},
                     "speedup": round(t1 / tf, 3),
                     "roofline": issue_roofline(
                         measured_instructions("k_fused_plane_wave.md", prec), win_ms[0],
                         int(wins[0]), torch.cuda.get_device_properties(dev).multi_processor_count),
                     "status": sim.diagnostics("electron").status}
        sim.close()
        del sim
    torch.cuda.synchronize()
    Q.qp_destroy(ctx)
    return out


# the step kernel's sources, and the unit that picks its launch (grid shape,
# cooperative or not)
STEP_SOURCES = ("qp_step.cuh", "qp_device.cuh", "qp_mixed.cuh", "qp_df.h", "qp_internal.h",
                "qp_kernels.h", "qp_step_fp64.cu", "qp_step_mixed.cu", "qp_kernels.cu")


def kernel_source_id() -> str:
    """Hash of the sources and build flags the step kernel is compiled from
    (the ncu summaries under profiles/ name the one they were taken on)."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1311_1107_gb300", "csrc")
    for f in STEP_SOURCES:
        h.update(f.encode())
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    for extra in (("include", "qedpic.h"), ("paper_1311_1107_gb300", "build.py")):
        with open(os.path.join(ROOT, *extra), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def measured_traffic(profile: str, precision: str):
    """DRAM bytes per k_step launch from the committed ncu summary of the
    workload, when it was taken on the current kernel sources; None
    otherwise (the counters no longer describe the kernel).  Returns
    (read, write, algorithmic): `algorithmic` is the model's bytes per
    launch of the captured launches when the summary states them (a capture
    of a smaller case of the workload), else None."""
    import re
    if profile is None:
        return None
    path = os.path.join(PROFILES, profile)
    if not os.path.exists(path):
        return None
    sid = kernel_source_id()
    pat = re.compile(r"^traffic, (\w+): read (\d+) B, write (\d+) B per launch"
                     r"(?:, algorithmic (\d+) B per launch)?, kernel source ([0-9a-f]{12})")
    with open(path) as f:
        for line in f:
            m = pat.match(line.strip())
            if m and m.group(1) == precision and m.group(5) == sid:
                alg = int(m.group(4)) if m.group(4) else None
                return int(m.group(2)), int(m.group(3)), alg
    return None


SM_MAX_MHZ = 2070.0     # GB300's maximum SM clock
ISSUE_PER_SM_CYCLE = 4  # warp instructions an SM issues a cycle (4 schedulers)


def measured_instructions(profile: str, precision: str):
    """Warp instructions of one fused window from the committed ncu summary,
    when it was taken on the current step-kernel sources; else None."""
    import re
    path = os.path.join(PROFILES, profile)
    if not os.path.exists(path):
        return None
    sid = kernel_source_id()
    pat = re.compile(r"^instructions, (\w+): (\d+) warp instructions per window, "
                     r"kernel source ([0-9a-f]{12})")
    with open(path) as f:
        for line in f:
            m = pat.match(line.strip())
            if m and m.group(1) == precision and m.group(3) == sid:
                return int(m.group(2))
    return None


def issue_roofline(instructions, window_ms, windows, sms):
    """The fused window's bound: instruction issue (it keeps the particles in
    registers; its DRAM traffic is negligible).  achieved = warp instructions
    of k_fused in one window (ncu) / the window's device time (CUDA events
    around its launches); peak = SMs x 4 schedulers x the maximum SM clock."""
    peak = sms * ISSUE_PER_SM_CYCLE * SM_MAX_MHZ * 1e6 / 1e9
    out = {"kernel": "k_fused", "bound": "alu", "unit": "G warp-instructions/s",
           "peak": round(peak, 1),
           "peak_source": f"{sms} SMs x {ISSUE_PER_SM_CYCLE} warp instructions a cycle x "
                          f"{SM_MAX_MHZ:.0f} MHz",
           "window_us": round(window_ms * 1e3 / max(windows, 1), 2), "achieved": None,
           "frac": None, "instructions_per_window": instructions}
    if instructions and window_ms > 0:
        achieved = instructions / (window_ms / max(windows, 1) * 1e-3) / 1e9
        out["achieved"] = round(achieved, 2)
        out["frac"] = round(achieved / peak, 4)
    return out


def roofline(res, dims, pairs, hbm_peak, peak_kind, traffic=None):
    """Roofline of k_step (the only kernel of a step): algorithmic bytes of
    all lepton and photon slot-steps and appended particles in the timed
    steps, over the summed k_step device time (CUDA events on its stream).
    traffic: (read, write, algorithmic) DRAM bytes per launch from an ncu
    capture (measured_traffic), or None.  A capture of a smaller case of the
    workload states the algorithmic bytes of its launches; its traffic is
    scaled to these launches by the ratio of algorithmic bytes (the traffic
    of a launch grows with the slots it steps and the particles it
    appends)."""
    lep_b, pho_b, new_b = species_bytes(dims, pairs)
    nbytes = (res["lep_slots"] * lep_b + res["pho_slots"] * pho_b
              + res.get("dead_slots", 0) * DEAD_B
              + (res["photons_added"] + 2 * res["pairs_added"]) * new_b)
    t_ms = res["kernel_ms"][0]
    n = max(res["launches"][0], 1)
    achieved = nbytes / (t_ms * 1e-3) / 1e9
    rw, scale = None, None
    if traffic:
        rd, wr, alg = traffic
        scale = (nbytes / n) / alg if alg else 1.0
        rw = [round(rd * scale), round(wr * scale)]
    out = {"kernel": "k_step", "bound": "hbm", "achieved": round(achieved, 2), "peak": hbm_peak,
           "unit": "GB/s", "frac": round(achieved / hbm_peak, 4),
           "traffic": sum(rw) if rw else None,
           "traffic_read_write": rw,
           "bytes_per_launch": round(nbytes / n), "avg_launch_us": round(t_ms * 1e3 / n, 3),
            "bytes_model": f"{lep_b} B per lepton slot-step, {pho_b} B per photon slot-step, "
                           f"{DEAD_B} B per decayed-photon slot (tau read), "
                           f"{new_b} B per appended particle",
            "peak_source": ("measured hbm_gbs, MEASURED_PEAKS.json" if peak_kind == "measured"
                            else "fallback 6.8 TB/s")}
    if traffic and traffic[2]:
        out["traffic_scaled"] = (f"from a smaller capture of the workload: x{scale:.3f}, "
                                 "the ratio of algorithmic bytes per launch")
    return out


def e2e_bytes(before, after, rows):
    """Bytes moved by one qp_step_host call: in, every array (`rows` per
    species) of the slots live before the step and the count; back, those
    slots without their weight row (a step writes the weights of appended
    particles only), the appended slots with every row, and the count."""
    h2d = sum(b * 8 * r + 8 for b, r in zip(before, rows))
    d2h = sum(b * 8 * (r - 1) + (a - b) * 8 * r + 8 for b, a, r in zip(before, after, rows))
    return h2d, d2h


def e2e(w, precision, steps, dev, warmup=3):
    """End to end through the public API with the state in host memory: every
    step is one qp_step_host call, which copies the live particles and
    counts from pinned host blocks to the device, runs the step, reads the
    new counts back and copies the new state back into the host blocks
    (and synchronises).  The bytes are the arrays of the live slots each
    way (back: without the weights of the slots live before the step, which
    a step does not change) plus the counts.  `warmup` untimed calls first
    (the first one allocates the context's pinned counts and look-back
    scratch), then the state is back at the initial one."""
    import torch

    from paper_1311_1107_gb300 import qedpic as Q
    from paper_1311_1107_gb300.sim import Simulation, stream_handle
    from paper_1311_1107_gb300.workloads import LAMBDA_M

    ctx = Q.qp_init_tables(LAMBDA_M, dev)
    sim = Simulation(w, precision=precision, ctx=ctx, device=dev, track_chi=False)
    names = ("electron", "positron", "photon")
    host = {n: torch.empty(sim.species[n].block.shape, dtype=torch.float64, pin_memory=True)
            for n in names}
    rows = {n: host[n].shape[0] for n in names}
    stream = torch.cuda.current_stream()
    st = stream_handle(stream)

    def initial_states():
        sim.load_initial()
        live = sim.live_counts()
        for n in names:
            sim.species[n].copy_state(host[n], live[n], False, st)
        torch.cuda.synchronize()
        return sim.host_states(host, live)

    states = initial_states()
    for _ in range(warmup):
        sim.run_host(states, 1, stream)
    states = initial_states()
    counts = [[int(states[k].count) for k in range(3)]]
    t0 = time.perf_counter()
    for _ in range(steps):
        sim.run_host(states, 1, stream)
        counts.append([int(states[k].count) for k in range(3)])
    wall = time.perf_counter() - t0
    torch.cuda.synchronize()
    r = [rows[n] for n in names]
    total_slots = sum(sum(c) for c in counts[:-1])
    h2d = d2h = 0
    for before, after in zip(counts[:-1], counts[1:]):
        i, o = e2e_bytes(before, after, r)
        h2d += i
        d2h += o
    Q.qp_destroy(ctx)
    return {"value": round(total_slots / wall, 1), "unit": UNIT,
            "h2d_bytes_per_step": int(h2d / steps), "d2h_bytes_per_step": int(d2h / steps),
            "steps": steps, "precision": precision,
            "api": "qp_step_host: host state copied in, stepped, copied back, one call a step"}


# ----------------------------------------------------------------------------- serving

def serving(dev, n_requests: int, n_max: float, load: float = 0.7):
    """Serve a stream of beam-collision requests (electron counts log-uniform
    in [1e3, n_max], gamma U[1000, 5000], a0 U[50, 500], steps U[200, 2000],
    seeds = ids) with Poisson arrivals.  The arrival rate is set so that the
    offered load is `load` of the batched throughput measured on the first
    8 requests served together (calibration, not timed).  Request payloads
    (initial electrons) are generated before the clock starts, as a client
    would send them."""
    import torch

    from paper_1311_1107_gb300 import qedpic as Q
    from paper_1311_1107_gb300 import workloads as W
    from paper_1311_1107_gb300.serve import ServingEngine

    reqs = W.serving_requests(n_requests=n_requests, arrival_rate=1.0, seed=0, n_max=n_max)
    payloads = {r["id"]: W.serving_request_workload(r, 8) for r in reqs}
    eng = ServingEngine(max_slots=Q.QP_MAX_BATCH, arena_bytes=96 << 30, graph_steps=8,
                        device=dev)
    try:
        cal_reqs = [dict(r, arrival_s=0.0) for r in reqs[:8]]
        cal = eng.run(cal_reqs, payloads)
        per_es = cal["particle_steps"] / sum(r["n"] * r["n_steps"] for r in cal_reqs)
        mean_work = per_es * float(np.mean([r["n"] * r["n_steps"] for r in reqs]))
        lam = load * cal["throughput"] / mean_work
        eng.max_concurrent = 0
        out = eng.run(reqs, payloads, time_scale=1.0 / lam)
    finally:
        eng.close()
    torch.cuda.synchronize(dev)
    lat = np.array([r["latency_s"] for r in out["results"]])
    return {
        "requests": n_requests, "completed": len(out["results"]),
        "throughput": round(out["throughput"], 1), "unit": UNIT,
        "p50_ms": round(float(np.percentile(lat, 50)) * 1e3, 2),
        "p99_ms": round(float(np.percentile(lat, 99)) * 1e3, 2),
        "arrival_rate_per_s": round(lam, 3), "offered_load": load,
        "calibration_throughput": round(cal["throughput"], 1),
        "makespan_s": round(out["makespan_s"], 2), "max_concurrent": out["max_concurrent"],
        "particle_steps": int(out["particle_steps"]), "graph_steps": 8, "precision": "mixed",
        "config": (f"{n_requests} requests: n_e log-uniform [1e3, {n_max:.0e}], gamma U[1000, 5000], "
                   "a0 U[50, 500], steps U[200, 2000], seeds 0.., Poisson arrivals; photon and "
                   "pair buffers 8 n_e; mixed path, CUDA graphs of 8 shared launches"),
    }


def serving_arm(args):
    import torch
    torch.cuda.set_device(0)
    n_req = args.requests or 256
    n_max = args.serving_nmax or 1e6
    clocks = ClockSampler(0)
    clocks.start()
    res = serving(0, n_req, n_max)
    clk = clocks.stop()
    line = {"metric": "serving: request latency and throughput (continuous batching)",
            "value": res["throughput"], "unit": UNIT, "n_gpus": 1, "steps": None,
            "warmup": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64 (mixed path)", "data": "synthetic",
            "config": {"workload": res["config"]}, "serving": res, "clocks": clk}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- CPU oracle

def oracle_sample(w, n_sample: int, n_steps: int, photons_per_electron: int = 256,
                  part=(0, 1), warmup: int = 0):
    """Time the CPU oracle (single thread) on a bounded sample of the
    workload: n_sample electrons (evenly spaced slots, each with its own
    random stream) for n_steps steps, after `warmup` untimed steps.
    part = (k, P): only the k-th of P contiguous parts of the sample (one
    process of an all-core run)."""
    import oracle as O
    from tests.parity import oracle_field

    n_all = len(w["electrons"]["x"])
    idx = np.linspace(0, n_all - 1, min(n_sample, n_all)).astype(np.int64)
    k, P = part
    idx = np.array_split(idx, P)[k]
    sub = {kk: np.asarray(v)[idx] for kk, v in w["electrons"].items()}
    dims = w["dims"]
    el = O.Species.from_arrays(sub, len(idx) * 4 + 64, dims, track=False, ids=idx)
    tau = np.zeros(n_all)
    O.lib().or_init_tau(int(w["params"]["seed"]), O.ELECTRON, tau.ctypes.data_as(O.C.c_void_p), 0,
                        n_all)
    el.tau[:len(idx)] = tau[idx]
    po = O.Species(len(idx) * 4 + 64, dims, track=False)
    ph = O.Species(len(idx) * photons_per_electron + 64, dims, track=False)
    O.tables()
    sim = O.Sim(oracle_field(w["field"]), w["params"], electrons=el, positrons=po, photons=ph)
    if warmup:
        sim.run(warmup)
    slots = 0
    t0 = time.perf_counter()
    for _ in range(n_steps):
        slots += el.n + po.n + ph.n
        sim.run(1)
    dt = time.perf_counter() - t0
    return slots, dt, len(idx)


def _oracle_part(args):
    """One process of an all-core oracle run (module level: spawn start)."""
    spec, n_sample, n_steps, ppe, k, P, warmup = args
    w = workload(*spec)
    return oracle_sample(w, n_sample, n_steps, ppe, (k, P), warmup)


def oracle_all_cores(spec, n_sample: int, n_steps: int, ppe: int, procs: int, warmup: int = 0):
    """The same sample split over `procs` processes (one per host core; each
    steps its part of the electrons with the oracle as it stands).  Returns
    (slot-steps, seconds of the slowest process, electrons)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    jobs = [(spec, n_sample, n_steps, ppe, k, procs, warmup) for k in range(procs)]
    with ctx.Pool(procs) as pool:
        parts = pool.map(_oracle_part, jobs)
    return (sum(p[0] for p in parts), max(p[1] for p in parts), sum(p[2] for p in parts))


CPU_BASELINE_SECONDS = 18.0


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(w, spec, args):
    """The oracle on about CPU_BASELINE_SECONDS of the same workload, on one
    core and on every host core (one process per core, the sample split
    between them): a short calibration sets how many evenly spaced electrons
    the timed sample steps (at most all of them, for the timed number of
    steps)."""
    collision = spec[0] == "collision"
    ppe = 256 if collision else 16
    steps = min(args.steps, 200)
    slots_c, dt_c, _ = oracle_sample(w, 2048, min(steps, 20), ppe)
    # the collision's later steps (more photons) cost more than its first
    seconds = CPU_BASELINE_SECONDS * (0.4 if collision else 1.0)
    target = seconds * slots_c / max(dt_c, 1e-6)  # particle-steps
    n_all = len(w["electrons"]["x"])
    n = int(min(n_all, max(1024, target / steps)))
    job_steps = max(args.steps, int(w["params"].get("n_steps", args.steps)))
    if n == n_all:  # every electron: more steps, up to the workload's own
        steps = int(min(job_steps, max(steps, target / n_all)))
    slots, dt, n1 = oracle_sample(w, n, steps, ppe)
    cores = host_cores()
    one = {"value": round(slots / dt, 1), "unit": UNIT, "cores": 1,
           "sample": f"{n1} electrons (evenly spaced slots) for {steps} steps, {dt:.1f} s"}
    if cores <= 1:
        return dict(one, kind="oracle")
    # all cores: about the same seconds of work per process; once every
    # electron is in the sample, more of the workload's steps
    n_all_cores = int(min(n_all, n * cores))
    steps_a = steps
    if n_all_cores == n_all:
        total = cores * slots / max(dt, 1e-6) * seconds
        steps_a = int(min(job_steps, max(steps, total / n_all)))
    slots_a, dt_a, na = oracle_all_cores(spec, n_all_cores, steps_a, ppe, cores)
    return {"value": round(slots_a / dt_a, 1), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{na} electrons (evenly spaced slots) split over {cores} processes "
                      f"(one per host core) for {steps_a} steps of the same workload, FP64 "
                      f"oracle, slowest process {dt_a:.1f} s",
            "one_core": one}


# ----------------------------------------------------------------------------- arms

def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as D
        torch.cuda.set_device(local)
        D.init_process_group("nccl")
        dist = D
    return world, rank, local, dist


def reference_arm(args):
    world, rank, _, dist = dist_setup(args)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    if args.workload in ("refill", "pic", "coalesce"):
        print(json.dumps({"impl": "reference",
                          "unavailable": "the oracle arm times the foil, collision, plane and "
                                         "fused (plane-wave) workloads"}), flush=True)
        if dist:
            dist.destroy_process_group()
        return
    spec = (args.workload, 0, args.start_step, args.collision_n)
    w = workload(*spec)
    cores = args.ref_cores or host_cores()
    per_core = 2048 if args.workload != "collision" else 512
    n_sample = per_core * cores
    ppe = 256 if args.workload == "collision" else 16
    slots, dt, n = oracle_all_cores(spec, n_sample, args.steps, ppe, cores, args.warmup)
    v = slots / dt
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 1), "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["name"], "sample": f"{n} electrons"},
            "cpu_baseline": {"value": round(v, 1), "unit": UNIT, "cores": cores,
                             "kind": "oracle",
                             "sample": f"{n} evenly spaced electrons of the workload split "
                                       f"over {cores} processes (one per host core), "
                                       f"{args.warmup} untimed + {args.steps} timed steps"},
            "e2e": {"value": round(v, 1), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def leg(w, args, dev, dist, flush, ids, profile, hbm_peak, peak_kind):
    """Mixed and FP64 paths on one workload: throughput over ranks, the
    roofline of each and the launch count."""
    from paper_1311_1107_gb300.shard import aggregate
    dims = w["dims"]
    pairs = bool(w["params"].get("pairs", False))
    mixed = run_path(w, "mixed", args.steps, args.warmup, dev, dist, flush, ids)
    fp64 = run_path(w, "fp64", args.steps, args.warmup, dev, dist, flush, ids)
    out = {}
    for name, res in (("mixed", mixed), ("fp64", fp64)):
        t_ms, slots = aggregate(sum(res["step_ms"]), res["lep_slots"] + res["pho_slots"], dist,
                                f"cuda:{dev}")
        out[name] = {
            "value": round(slots / (t_ms * 1e-3), 1), "unit": UNIT,
            "ms_per_step": round(t_ms / args.steps, 4),
            "roofline": roofline(res, dims, pairs, hbm_peak, peak_kind,
                                 measured_traffic(profile, name)),
            "final_live": res["final_live"], "status": res["status"],
            "launches": int(sum(res["launches"])),
            "decayed_photon_slot_steps": res["dead_slots"], "pair_drops": res["pair_drops"],
        }
    for res in (mixed, fp64):
        res["sim"].close()
        del res["sim"]
    import torch
    from paper_1311_1107_gb300 import qedpic as Q
    torch.cuda.synchronize()
    for res in (mixed, fp64):
        Q.qp_destroy(res["ctx"])
    torch.cuda.empty_cache()
    return out


def ours_arm(args):
    import torch

    from paper_1311_1107_gb300.shard import shard_ids

    world, rank, local, dist = dist_setup(args)
    dev = local
    torch.cuda.set_device(dev)
    # every rank steps its own shard of one population of `world` copies of
    # the workload: the same initial state, disjoint particle ids (its own
    # random streams), no exchange between ranks
    spec = (args.workload, 0, args.start_step, args.collision_n)
    w = workload(*spec)
    ids = shard_ids(world * len(w["electrons"]["x"]), rank, world, w["capacity"])
    hbm_peak, peak_kind = peaks()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{dev}")
    profile = {"foil": "k_step_foil2d.md", "collision": "k_step_collision.md"}.get(
        args.workload, "k_step_" + args.workload + ".md")
    if args.workload in ("refill", "pic"):
        profile = None  # more kernels than k_step a step: no k_step traffic line

    clocks = ClockSampler(dev)
    clocks.start()
    main_leg = leg(w, args, dev, dist, flush, ids, profile, hbm_peak, peak_kind)
    # the beam collision at full size (1e7 e-, 1e8-slot buffers, the steps
    # around the pulse peak): the many-particle state of the HBM roofline
    coll = None
    if world == 1 and args.workload == "foil" and not args.no_collision:
        wc = workload("collision", 0, args.start_step, args.collision_n)
        idc = shard_ids(len(wc["electrons"]["x"]), 0, 1, wc["capacity"])
        c = leg(wc, args, dev, dist, flush, idc, "k_step_collision.md", hbm_peak, peak_kind)
        coll = {"workload": wc["name"], "value": c["mixed"]["value"], "unit": UNIT,
                "ms_per_step": c["mixed"]["ms_per_step"], "roofline": c["mixed"]["roofline"],
                "final_live": c["mixed"]["final_live"],
                "decayed_photon_slot_steps": c["mixed"]["decayed_photon_slot_steps"],
                "fp64": {k: c["fp64"][k] for k in ("value", "ms_per_step", "roofline",
                                                   "final_live")},
                "mixed_over_fp64": round(c["mixed"]["value"] / c["fp64"]["value"], 3),
                "status": {"mixed": c["mixed"]["status"], "fp64": c["fp64"]["status"]},
                "launches": c["mixed"]["launches"] + c["fp64"]["launches"]}
        del wc
    # the same foil with its fields refilled from the pulse before every step
    # (qp_fill_yee2d: two more launches a step, inside the timed steps)
    refill = None
    if world == 1 and args.workload == "foil" and not args.no_collision:
        from paper_1311_1107_gb300 import workloads as W
        wr = W.laser_on_foil(seed=0, refill=True)
        r = leg(wr, args, dev, dist, flush, ids, "k_step_foil2d.md", hbm_peak, peak_kind)
        refill = {"workload": wr["name"], "value": r["mixed"]["value"], "unit": UNIT,
                  "ms_per_step": r["mixed"]["ms_per_step"],
                  "roofline": dict(r["mixed"]["roofline"], traffic=None,
                                   traffic_read_write=None),
                  "fp64": {k: r["fp64"][k] for k in ("value", "ms_per_step")},
                  "status": {"mixed": r["mixed"]["status"], "fp64": r["fp64"]["status"]}}
        del wr
    # the same foil as a PIC cycle: the grid's own fields advanced by the
    # Yee solver with the electrons' current around every QED step
    pic = None
    if world == 1 and args.workload == "foil" and not args.no_collision:
        from paper_1311_1107_gb300 import workloads as W
        wp = W.laser_on_foil(seed=0, pic=True)
        r = leg(wp, args, dev, dist, flush, ids, "k_step_foil2d.md", hbm_peak, peak_kind)
        pic = {"workload": wp["name"], "value": r["mixed"]["value"], "unit": UNIT,
               "ms_per_step": r["mixed"]["ms_per_step"],
               "roofline": dict(r["mixed"]["roofline"], traffic=None, traffic_read_write=None),
               "fp64": {k: r["fp64"][k] for k in ("value", "ms_per_step")},
               "status": {"mixed": r["mixed"]["status"], "fp64": r["fp64"]["status"]}}
        del wp
    fused = None
    if world == 1 and args.workload == "foil" and not args.no_collision:
        fused = fused_leg(dev, flush, args.warmup)
    serv = None
    if rank == 0 and world == 1 and not args.no_serving:
        serv = serving(dev, args.requests or 256, args.serving_nmax or 1e6)
    clk = clocks.stop()
    v_mixed, v_fp64 = main_leg["mixed"]["value"], main_leg["fp64"]["value"]
    if rank == 0:
        e2e_res = None
        if not args.no_e2e:
            e2e_res = e2e(w, "mixed", min(args.e2e_steps, args.steps), dev,
                          max(args.warmup, 1))
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            cpu = cpu_baseline(w, spec, args)
        launches = main_leg["mixed"]["launches"]
        line = {
            "metric": METRIC, "value": v_mixed, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": main_leg["mixed"]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64 (mixed path)",
            "data": "synthetic",
            "config": {"workload": w["name"], "precision": "mixed",
                       "l2": "flushed between timed steps (256 MB write)",
                       "particle_steps": "live slots of e-, e+ and photons at each step start, "
                                         "decayed photons (tau < 0) left out",
                       "steps_timed": "steps 0..K-1 of the job from the initial state"
                       if args.workload != "collision" else
                       f"K steps from step {wc_start(args)}",
                       "final_live": main_leg["mixed"]["final_live"],
                       "parallelism": f"shards x{world} (disjoint particle ids per rank, "
                                      "no exchange)"},
            "fp64": {"value": v_fp64, "unit": UNIT,
                     "ms_per_step": main_leg["fp64"]["ms_per_step"], "dtype": "f64",
                     "roofline": main_leg["fp64"]["roofline"],
                     "mixed_over_fp64": round(v_mixed / v_fp64, 3),
                     "final_live": main_leg["fp64"]["final_live"]},
            "roofline": main_leg["mixed"]["roofline"],
            "collision": coll, "refill": refill, "pic": pic, "fused": fused,
            "cpu_baseline": cpu, "e2e": e2e_res, "gpu_launches": launches, "serving": serv,
            "clocks": clk,
            "status": {"mixed": main_leg["mixed"]["status"], "fp64": main_leg["fp64"]["status"]},
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def wc_start(args) -> int:
    return 980 if args.start_step is None else args.start_step


def fused_arm(args):
    """--workload fused: the fused plane-wave leg alone (one JSON line)."""
    import torch
    torch.cuda.set_device(0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda:0")
    clocks = ClockSampler(0)
    clocks.start()
    res = fused_leg(0, flush, args.warmup)
    clk = clocks.stop()
    line = {"metric": "fused steps: particle-steps/s, one launch a step vs fused windows",
            "value": res["mixed"]["fused"]["value"], "unit": UNIT, "n_gpus": 1, "steps": 1000,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64 (mixed path)", "data": "synthetic",
            "config": {"workload": res["workload"]}, "fused": res, "clocks": clk}
    print(json.dumps(line), flush=True)


COALESCE_STEPS = 30


def coalesce_arm(args):
    """--workload coalesce: the photons of the beam collision after its
    window (collision-n electrons, steps from start-step), compacted and
    coalesced; K timed repetitions, each on a fresh copy of the photons."""
    import torch

    from paper_1311_1107_gb300 import qedpic as Q
    from paper_1311_1107_gb300 import workloads as W
    from paper_1311_1107_gb300.sim import Simulation

    torch.cuda.set_device(0)
    w = workload("collision", 0, args.start_step, args.collision_n or 2e6)
    ctx = Q.qp_init_tables(W.LAMBDA_M, 0)
    sim = Simulation(w, precision="mixed", ctx=ctx, track_chi=False)
    sim.run(COALESCE_STEPS)
    torch.cuda.synchronize()
    ph = sim.species["photon"]
    n = ph.count()
    keep = ph.block[:, :n].clone()
    sig = W.length(2e-6)
    # a box over the beam's 4 sigma, 8 energy bins an octave, 8 direction bins
    x0 = float(ph.t["x"][:n].min()) - 1.0
    box = (x0, -4 * sig, -4 * sig, 8 * sig / 32, 8 * sig / 32, 8 * sig / 32)
    p = Q.coalesce_params(box, (64, 32, 32), 8, 8, 3, seed=1, step=sim.step_index)
    stream = torch.cuda.current_stream()
    times, stats = [], None
    for rep in range(args.warmup + args.steps):
        ph.block[:, :n].copy_(keep)
        ph.n_live.fill_(n)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        Q.qp_coalesce_photons(ctx, ph.handle, p, None, stats=False)
        b.record(stream)
        torch.cuda.synchronize()
        if rep >= args.warmup:
            times.append(a.elapsed_time(b))
    stats = Q.qp_coalesce_photons(ctx, ph.handle, None)  # compaction of the result
    ms = float(np.median(times))
    line = {"metric": "super-photon coalescence: photons/s", "value": round(n / (ms * 1e-3), 1),
            "unit": "photons/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"photons of {w['name']} after {COALESCE_STEPS} steps",
                       "photons": n, "after": stats["n_after"], "grid": "64x32x32 cells",
                       "bins": "8 energy bins an octave, 8 direction bins"}}
    print(json.dumps(line), flush=True)
    sim.close()
    Q.qp_destroy(ctx)


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    elif args.workload == "serving":
        serving_arm(args)
    elif args.workload == "fused":
        fused_arm(args)
    elif args.workload == "coalesce":
        coalesce_arm(args)
    else:
        ours_arm(args)


if __name__ == "__main__":
    main()
