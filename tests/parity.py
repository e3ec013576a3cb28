"""Helpers of the GPU parity tests: run one seeded workload through the CUDA
path (via the C ABI) and through the CPU oracle, and compare."""
from __future__ import annotations

import numpy as np

import oracle as O

SPECIES = ("electron", "positron", "photon")
ORACLE_KIND = {"electron": O.ELECTRON, "positron": O.POSITRON, "photon": O.PHOTON}
FIELDS = ("x", "y", "z", "ux", "uy", "uz", "tau", "w")


def oracle_field(desc):
    k = desc["kind"]
    if k == "plane":
        return O.plane_field(desc["a0"])
    if k == "gaussian":
        return O.gaussian_field(desc["a0"], desc["w0"], desc["tau_fwhm"], desc["x_focus"],
                                desc["t_focus"])
    if k == "uniform_b":
        return O.uniform_b_field(desc["b0"])
    if k == "yee2d":
        return O.yee2d_field(desc["comps"], desc["dx"], desc["dy"], desc.get("x0", 0.0),
                             desc.get("y0", 0.0))
    f = O.Field()
    f.kind = O.FIELD_NONE
    return f


def run_oracle(workload, n_steps, sample=None, extra=None):
    """Run the oracle on a workload.  sample: optional slot indices of the
    electrons to keep (each keeps its random stream).  extra: optional dict
    species -> arrays of initial positrons/photons (with their own tau)."""
    dims = workload["dims"]
    cap = dict(workload["capacity"])
    el_arr = workload["electrons"]
    n_all = len(el_arr["x"])
    tau_all = np.zeros(max(n_all, 1))
    O.lib().or_init_tau(int(workload["params"]["seed"]), O.ELECTRON,
                        tau_all.ctypes.data_as(O.C.c_void_p), 0, n_all)
    if sample is None:
        el = O.Species.from_arrays(el_arr, cap["electron"], dims)
        el.tau[:n_all] = tau_all[:n_all]
    else:
        sample = np.asarray(sample)
        sub = {k: np.asarray(v)[sample] for k, v in el_arr.items()}
        el = O.Species.from_arrays(sub, len(sample) * 64 + 64, dims, ids=sample)
        el.tau[:len(sample)] = tau_all[sample]
        cap = {"electron": el.cap, "positron": len(sample) * 64 + 64,
               "photon": len(sample) * 4096}
    po = O.Species(max(cap["positron"], 1), dims)
    ph = O.Species(max(cap["photon"], 1), dims)
    if cap["positron"] == 0:
        po.cap = 0
    if cap["photon"] == 0:
        ph.cap = 0
    for name, sp in (("positron", po), ("photon", ph)):
        if extra and name in extra:
            arr = extra[name]
            n = len(arr["x"])
            for nm in O.Species.NAMES:
                if getattr(sp, nm) is not None and nm in arr:
                    getattr(sp, nm)[:n] = arr[nm]
            sp.n = n
    sim = O.Sim(oracle_field(workload["field"]), workload["params"], electrons=el, positrons=po,
                photons=ph)
    sim.run(n_steps)
    return sim, {"electron": el, "positron": po, "photon": ph}


def oracle_arrays(sp):
    return {nm: (None if getattr(sp, nm) is None else getattr(sp, nm)[:sp.n].copy())
            for nm in FIELDS}


def rel_err(a, b, floor):
    """|a - b| / max(|b|, floor), elementwise."""
    return np.abs(a - b) / np.maximum(np.abs(b), floor)


def compare_species(gpu: dict, ora: dict, rtol, pos_atol, label=""):
    """Slot-by-slot comparison of one species' live state; returns the max
    relative momentum error seen."""
    n = len(ora["x"])
    assert len(gpu["x"]) == n, f"{label}: live count gpu {len(gpu['x'])} oracle {n}"
    if n == 0:
        return 0.0
    umag = np.sqrt(ora["ux"] ** 2 + ora["uy"] ** 2 + ora["uz"] ** 2)
    floor = np.maximum(umag, 1.0)
    worst = 0.0
    for c in ("ux", "uy", "uz"):
        e = np.abs(gpu[c] - ora[c]) / floor
        worst = max(worst, float(e.max()))
        assert e.max() <= rtol, f"{label} {c}: max rel err {e.max():.3g} at slot {e.argmax()}"
    for c in ("x", "y", "z"):
        if ora[c] is None:
            continue
        e = np.abs(gpu[c] - ora[c])
        assert e.max() <= pos_atol, f"{label} {c}: max abs err {e.max():.3g} at slot {e.argmax()}"
    # optical depth: alive/dead must agree exactly, values within tolerance
    assert np.array_equal(gpu["tau"] < 0, ora["tau"] < 0), f"{label}: dead photons differ"
    e = np.abs(gpu["tau"] - ora["tau"]) / np.maximum(np.abs(ora["tau"]), 1.0)
    assert e.max() <= rtol, f"{label} tau: max err {e.max():.3g} at slot {e.argmax()}"
    np.testing.assert_array_equal(gpu["w"], ora["w"])
    return worst
