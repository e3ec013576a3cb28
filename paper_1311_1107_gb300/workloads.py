"""Seeded synthetic inputs for the QED particle step.

Initial particle states, laser/field descriptions and the fixed Yee field
snapshot of the laser-on-foil case.  This module holds none of the step's
arithmetic: it only draws initial conditions (numpy ``default_rng``) and
evaluates the input laser field on a grid.  Both the CUDA path and the CPU
oracle consume what it returns.

Units are the library's normalised units at the reference wavelength
(0.8 um): time in 1/omega, length in c/omega, momentum in m c, fields in
m c omega / e.  ``T_PERIOD = 2 pi`` is one laser period.
"""
from __future__ import annotations

import math

import numpy as np

LAMBDA_M = 0.8e-6
C_LIGHT = 299792458.0
OMEGA = 2.0 * math.pi * C_LIGHT / LAMBDA_M
T_PERIOD = 2.0 * math.pi
K_PER_M = 2.0 * math.pi / LAMBDA_M  # metres -> c/omega


def length(m: float) -> float:
    """Metres to normalised length (c/omega)."""
    return m * K_PER_M


def duration(s: float) -> float:
    """Seconds to normalised time (1/omega)."""
    return s * OMEGA


def _empty_species():
    return {k: np.zeros(0) for k in ("x", "y", "z", "ux", "uy", "uz", "w")}


# ----------------------------------------------------------------------------
# Single species against a plane wave (4096 e-, gamma 2000, a0 100, 1000 steps)
# ----------------------------------------------------------------------------

def plane_wave_collision(n: int = 4096, gamma: float = 2000.0, a0: float = 100.0,
                         n_steps: int = 1000, seed: int = 0):
    """All electrons at the origin moving along -x with the same gamma, head-on
    with a linearly polarised plane wave along +x.  FP64, Monte-Carlo only,
    photons tracked, no pairs."""
    p = math.sqrt(gamma * gamma - 1.0)
    el = {
        "x": np.zeros(n), "y": np.zeros(n), "z": np.zeros(n),
        "ux": np.full(n, -p), "uy": np.zeros(n), "uz": np.zeros(n),
        "w": np.ones(n),
    }
    return {
        "name": f"plane-wave collision: {n} e-, gamma {gamma:g}, a0 {a0:g}, {n_steps} steps",
        "dims": 3,
        "electrons": el,
        "field": {"kind": "plane", "a0": a0},
        "params": {"dt": T_PERIOD / 100.0, "n_steps": n_steps, "seed": seed, "chi_th": 0.0,
                   "photon_min_gamma": 2.0, "pairs": False, "max_emit": 8},
        "capacity": {"electron": n, "positron": 0, "photon": n * 256},
    }


# ----------------------------------------------------------------------------
# 2D laser-on-foil with a fixed Yee field snapshot
# ----------------------------------------------------------------------------

def gaussian_2d_snapshot(nx: int, ny: int, dx: float, dy: float, a0: float, w0: float,
                         tau_fwhm: float, x_focus: float, y_axis: float):
    """Lowest-order paraxial 2D Gaussian pulse along +x, polarised along y,
    evaluated at the instant its envelope peak sits at the focal plane.
    Returns Ex Ey Ez Bx By Bz (float32, shape (ny, nx)) on the Yee staggering
    Ex (i+1/2, j), Ey (i, j+1/2), Ez (i, j), Bx (i, j+1/2), By (i+1/2, j),
    Bz (i+1/2, j+1/2)."""
    zr = 0.5 * w0 * w0

    def ey(x, y):
        xi = x - x_focus
        q = xi / zr
        wr2 = 1.0 + q * q
        r2 = (y - y_axis) ** 2
        env = -r2 / (w0 * w0 * wr2) - 2.0 * math.log(2.0) * xi * xi / (tau_fwhm * tau_fwhm)
        amp = a0 * wr2 ** -0.25 * np.exp(env)
        phase = xi + r2 * xi / (2.0 * (xi * xi + zr * zr)) - 0.5 * np.arctan(q)
        return amp * np.cos(phase)

    ii = np.arange(nx, dtype=np.float64)
    jj = np.arange(ny, dtype=np.float64)
    X, Yh = np.meshgrid(ii * dx, (jj + 0.5) * dy)           # Ey node
    Xh, Yh2 = np.meshgrid((ii + 0.5) * dx, (jj + 0.5) * dy)  # Bz node
    Ey = ey(X, Yh).astype(np.float32)
    Bz = ey(Xh, Yh2).astype(np.float32)
    z = np.zeros((ny, nx), dtype=np.float32)
    return [z, Ey, z.copy(), z.copy(), z.copy(), Bz]


def laser_on_foil(nx: int = 2048, ny: int = 512, ppc: int = 8, a0: float = 200.0,
                  n_steps: int = 500, seed: int = 0, foil_cells: int = 32,
                  photon_capacity: int = 1 << 25, pair_capacity: int = 1 << 20,
                  refill: bool = False, pic: bool = False):
    """2048x512 grid, dx = lambda/32, a 1-lambda foil of electrons at
    n = 100 n_c, 8 per cell, Maxwellian 1 keV, in the fixed fields of a
    Gaussian pulse (a0 200, waist 3 lambda, 30 fs FWHM) whose peak sits at the
    foil front.  Sokolov damping below chi 1e-3, Monte-Carlo above.
    refill: the grid's E_y and B_z are refilled from the pulse before every
    step instead (qp_fill_yee2d); the pulse's peak reaches the foil front at
    mid-run; the grid starts empty.
    pic: the fields are the grid's own, advanced by the Yee solver with the
    electrons' current (qp_yee_advance_*, qp_deposit_current): the grid
    starts with the pulse of `refill` at the first step's time and the pulse
    then propagates, diffracts and meets the foil on the grid."""
    rng = np.random.default_rng(seed)
    dx = dy = T_PERIOD / 32.0
    i0 = nx // 2
    ncell = foil_cells * ny
    n = ncell * ppc
    ci = i0 + np.repeat(np.arange(foil_cells), ny * ppc)
    cj = np.tile(np.repeat(np.arange(ny), ppc), foil_cells)
    x = (ci + rng.random(n)) * dx
    y = (cj + rng.random(n)) * dy
    sigma_u = math.sqrt(1.0e3 / 510998.95)  # kT / m c^2 for 1 keV
    u = rng.normal(0.0, sigma_u, size=(3, n))
    w = np.full(n, 100.0 * dx * dy / ppc)
    el = {"x": x, "y": y, "ux": u[0], "uy": u[1], "uz": u[2], "w": w}
    w0, tau = length(3 * LAMBDA_M), duration(30e-15)
    dt = 0.95 * dx / math.sqrt(2.0)
    field = {"kind": "yee2d", "dx": dx, "dy": dy, "x0": 0.0, "y0": 0.0}
    if refill or pic:
        field["comps"] = [np.zeros((ny, nx), dtype=np.float32) for _ in range(6)]
        field["refill" if refill else "pic"] = {
            "a0": a0, "w0": w0, "tau_fwhm": tau, "x_focus": i0 * dx,
            "t_focus": (n_steps // 2) * dt, "y_axis": 0.5 * ny * dy}
    else:
        field["comps"] = gaussian_2d_snapshot(nx, ny, dx, dy, a0=a0, w0=w0, tau_fwhm=tau,
                                              x_focus=i0 * dx, y_axis=0.5 * ny * dy)
    return {
        "name": (f"2D laser-on-foil: {nx}x{ny} Yee grid, {n} e-, a0 {a0:g}, {n_steps} steps"
                 + (", fields refilled from the pulse every step" if refill else "")
                 + (", PIC fields (Yee solver and current deposition)" if pic else "")),
        "dims": 2,
        "electrons": el,
        "field": field,
        "params": {"dt": dt, "n_steps": n_steps, "seed": seed,
                   "chi_th": 1e-3, "photon_min_gamma": 2.0, "pairs": True, "max_emit": 8},
        "capacity": {"electron": n + pair_capacity, "positron": pair_capacity,
                     "photon": photon_capacity},
    }


# ----------------------------------------------------------------------------
# GeV beam against a Gaussian pulse, with pairs
# ----------------------------------------------------------------------------

def beam_collision(n: int = 10_000_000, gamma: float = 4000.0, spread: float = 0.05,
                   a0: float = 500.0, n_steps: int = 2000, seed: int = 0,
                   buffer: int = 100_000_000, sigma_m: float = 2e-6,
                   waist_m: float = 2e-6, fwhm_s: float = 30e-15):
    """Electron beam (Gaussian energy spread and Gaussian spatial profile)
    along -x, head-on with a 3D paraxial Gaussian pulse along +x; the pulse
    peak and the beam centre meet at the focus at mid-run."""
    rng = np.random.default_rng(seed)
    dt = T_PERIOD / 100.0
    t_meet = 0.5 * n_steps * dt
    sig = length(sigma_m)
    g = rng.normal(gamma, spread * gamma, size=n)
    g = np.maximum(g, 2.0)
    p = np.sqrt(g * g - 1.0)
    el = {
        "x": t_meet + rng.normal(0.0, sig, size=n),
        "y": rng.normal(0.0, sig, size=n),
        "z": rng.normal(0.0, sig, size=n),
        "ux": -p, "uy": np.zeros(n), "uz": np.zeros(n),
        "w": np.ones(n),
    }
    return {
        "name": (f"beam collision: {n} e-, gamma {gamma:g} +-{spread:.0%}, a0 {a0:g}, "
                 f"{n_steps} steps, {buffer} slot buffers"),
        "dims": 3,
        "electrons": el,
        "field": {"kind": "gaussian", "a0": a0, "w0": length(waist_m),
                  "tau_fwhm": duration(fwhm_s), "x_focus": 0.0, "t_focus": t_meet},
        "params": {"dt": dt, "n_steps": n_steps, "seed": seed, "chi_th": 1e-3,
                   "photon_min_gamma": 2.0, "pairs": True, "max_emit": 8},
        "capacity": {"electron": n + buffer, "positron": buffer, "photon": buffer},
    }


# ----------------------------------------------------------------------------
# Constant-B cascade of the paper's validation test (gamma 3000, B 7.48 MT)
# ----------------------------------------------------------------------------

def uniform_b_cascade(n: int = 1024, gamma: float = 3000.0, b_tesla: float = 7.48e6,
                      n_steps: int = 400, seed: int = 0, cap: int = 1 << 20):
    """Electrons with gamma 3000 perpendicular to a constant B = 7.48 MT."""
    me, qe = 9.1093837015e-31, 1.602176634e-19
    b0 = qe * b_tesla / (me * OMEGA)
    p = math.sqrt(gamma * gamma - 1.0)
    el = {"x": np.zeros(n), "y": np.zeros(n), "z": np.zeros(n),
          "ux": np.full(n, p), "uy": np.zeros(n), "uz": np.zeros(n), "w": np.ones(n)}
    period = 2.0 * math.pi * gamma / b0
    return {
        "name": f"constant-B cascade: {n} e-, gamma {gamma:g}, B {b_tesla:g} T",
        "dims": 3,
        "electrons": el,
        "field": {"kind": "uniform_b", "b0": b0},
        "params": {"dt": period / 200.0, "n_steps": n_steps, "seed": seed, "chi_th": 0.0,
                   "photon_min_gamma": 2.0, "pairs": True, "max_emit": 8},
        "capacity": {"electron": n + cap, "positron": cap, "photon": cap},
    }


# ----------------------------------------------------------------------------
# Serving stream: independent collision requests with Poisson arrivals
# ----------------------------------------------------------------------------

def serving_requests(n_requests: int = 256, arrival_rate: float = 100.0, seed: int = 0,
                     n_min: float = 1e3, n_max: float = 1e6):
    """Request descriptors: electron count log-uniform in [1e3, 1e6], gamma
    uniform in [1000, 5000], a0 uniform in [50, 500], steps uniform in
    [200, 2000], request seeds 0..255, Poisson arrival times (seed 0)."""
    rng = np.random.default_rng(seed)
    n_e = np.exp(rng.uniform(math.log(n_min), math.log(n_max), size=n_requests)).astype(np.int64)
    gam = rng.uniform(1000.0, 5000.0, size=n_requests)
    a0 = rng.uniform(50.0, 500.0, size=n_requests)
    steps = rng.integers(200, 2001, size=n_requests)
    gaps = rng.exponential(1.0 / arrival_rate, size=n_requests)
    arrival = np.cumsum(gaps) - gaps[0]
    return [
        {"id": i, "seed": i, "n": int(n_e[i]), "gamma": float(gam[i]), "a0": float(a0[i]),
         "n_steps": int(steps[i]), "arrival_s": float(arrival[i])}
        for i in range(n_requests)
    ]


def serving_request_workload(req: dict, capacity_factor: int = 8):
    """The particles and fields of one serving request: a beam collision with
    the request's count, energy, amplitude, step count and seed."""
    w = beam_collision(n=req["n"], gamma=req["gamma"], a0=req["a0"], n_steps=req["n_steps"],
                       seed=req["seed"], buffer=capacity_factor * req["n"])
    w["name"] = f"request {req['id']}: " + w["name"]
    return w
