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


def oracle_pulse(desc):
    rf = desc.get("refill")
    if not rf:
        return None
    return O.pulse2d(rf["a0"], rf["w0"], rf["tau_fwhm"], rf["x_focus"], rf["t_focus"],
                     rf["y_axis"])


def oracle_pic_start(sim, workload):
    """The oracle's grid of a PIC workload at its first step: the pulse at
    that time (E and B), the other components zero."""
    pc = workload["field"]["pic"]
    p = O.pulse2d(pc["a0"], pc["w0"], pc["tau_fwhm"], pc["x_focus"], pc["t_focus"], pc["y_axis"])
    for c in sim.field._keep:
        c[:] = 0.0
    O.fill_pulse2d(p, sim.field, sim.P.step * sim.P.dt)


def oracle_pic_steps(sim, n_steps, field_noise=0.0, noise_key=0):
    """PIC cycles of the oracle: B half step, the QED step, the leptons'
    current (FP64, rounded to the grid's float), B half step, E full step.
    field_noise: relative +-kick of every grid value after every cycle (a
    twin run's model of the device's FP32 solver arithmetic and unordered
    current sums, which the oracle's FP64 solver does not have)."""
    f = sim.field
    comps = f._keep
    dt = sim.P.dt
    rng = np.random.default_rng(1000 + noise_key) if field_noise else None
    for _ in range(n_steps):
        O.yee_advance_b(comps, f.dx, f.dy, 0.5 * dt)
        sim.run(1)
        J = [np.zeros(comps[0].shape) for _ in range(3)]
        for q, sp in ((-1.0, sim.sp[0]), (1.0, sim.sp[1])):
            if sp is not None and sp.n:
                O.deposit_current(sp, q, dt, J, f.dx, f.dy, f.x0, f.y0)
        O.yee_advance_b(comps, f.dx, f.dy, 0.5 * dt)
        O.yee_advance_e(comps, [j.astype(np.float32) for j in J], f.dx, f.dy, dt)
        if field_noise:
            for c in comps:
                c *= (1.0 + field_noise * rng.choice((-1.0, 1.0), size=c.shape)).astype(c.dtype)


def oracle_steps(sim, workload, n_steps, field_noise=0.0, noise_key=0):
    """n_steps of an oracle run; a workload with a refilled grid gets the
    oracle's own refill (from the pulse, FP64 rounded to float) before each
    step, a PIC workload the oracle's own solver and deposition (with
    field_noise, kicked after every cycle: see oracle_pic_steps)."""
    if workload["field"].get("pic"):
        oracle_pic_steps(sim, n_steps, field_noise, noise_key)
        return
    pulse = oracle_pulse(workload["field"])
    if pulse is None:
        sim.run(n_steps)
        return
    for _ in range(n_steps):
        O.fill_pulse2d(pulse, sim.field, sim.P.step * sim.P.dt)
        sim.run(1)


def run_oracle(workload, n_steps, sample=None, extra=None, kick=0.0, noise=0.0, noise_key=0,
               field_noise=0.0):
    """Run the oracle on a workload.  sample: optional slot indices of the
    electrons to keep (each keeps its random stream).  extra: optional dict
    species -> arrays of initial positrons/photons (with their own tau).
    kick: relative perturbation of the initial electron momenta (sign
    alternating with the slot); noise: relative +-kick of every lepton
    momentum after every step; field_noise (PIC workloads): relative +-kick
    of every grid value after every cycle.  All serve the twin run that
    measures how strongly each trajectory amplifies rounding-level
    differences."""
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
    if kick:
        n0 = el.n
        ids = np.arange(n0) if sample is None else np.asarray(sample)
        sign = np.where(ids % 2 == 0, 1.0, -1.0)
        for c in ("ux", "uy", "uz"):
            getattr(el, c)[:n0] *= 1.0 + kick * sign
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
    params = dict(workload["params"])
    if noise:
        params["noise"] = noise
        params["noise_key"] = noise_key
    sim = O.Sim(oracle_field(workload["field"]), params, electrons=el, positrons=po,
                photons=ph)
    if workload["field"].get("pic"):
        oracle_pic_start(sim, workload)
    oracle_steps(sim, workload, n_steps, field_noise, noise_key)
    return sim, {"electron": el, "positron": po, "photon": ph}


def run_oracle_from_state(workload, state, step, n_steps=1):
    """Restart the oracle from a saved state (dict species -> host arrays, as
    returned by DeviceSpecies.host()) at step index `step` and run n_steps.
    Optical depths come from the state; per-particle event counts start at 0."""
    dims = workload["dims"]
    cap = workload["capacity"]
    sps = {}
    for name in SPECIES:
        arr = state[name]
        n = len(arr["x"])
        sp = O.Species(max(cap[name], n, 1), dims)
        if cap[name] == 0:
            sp.cap = 0
        for nm in O.Species.NAMES:
            if getattr(sp, nm) is not None and nm in arr and n:
                getattr(sp, nm)[:n] = arr[nm]
        sp.n = n
        sps[name] = sp
    params = dict(workload["params"])
    params["step"] = int(step)
    sim = O.Sim(oracle_field(workload["field"]), params, electrons=sps["electron"],
                positrons=sps["positron"], photons=sps["photon"])
    oracle_steps(sim, workload, n_steps)
    return sim, sps


def oracle_arrays(sp):
    out = {nm: (None if getattr(sp, nm) is None else getattr(sp, nm)[:sp.n].copy())
           for nm in FIELDS}
    if sp.nemit is not None:
        out["nemit"] = sp.nemit[:sp.n].copy()
    if sp.chi is not None:
        out["chi"] = sp.chi[:sp.n].copy()
    return out


# chi below this is compared in absolute terms: its rates are ~1e-9 of the
# step's and an FP32 field tail may underflow where the FP64 one does not
CHI_FLOOR = 1e-6


def chi_report(gpu, ora, sel):
    """chi_e of the particles `sel`: the largest and median error relative to
    each particle's own chi (reported), and the largest absolute error over
    the largest chi of the population (bounded).  A field evaluated in FP32
    carries an absolute error of ~1e-7 of its amplitude and phase, so a
    particle near a node of the wave, where its own chi almost vanishes, can
    show a large relative error in a chi that has no weight in its rates;
    the rates, and so tau and the events, are compared on their own."""
    ec = chi_error(gpu, ora)
    if ec is None or not sel.any():
        return {}
    scale = max(float(np.max(np.abs(ora["chi"][sel]))), CHI_FLOOR)
    return {"chi_max": float(ec[sel].max()), "chi_median": float(np.median(ec[sel])),
            "chi_abs_over_max": float(np.max(np.abs(gpu["chi"][sel] - ora["chi"][sel]))) / scale}


def gamma_error(a, b):
    ga = np.sqrt(1.0 + a["ux"] ** 2 + a["uy"] ** 2 + a["uz"] ** 2)
    gb = np.sqrt(1.0 + b["ux"] ** 2 + b["uy"] ** 2 + b["uz"] ** 2)
    return np.abs(ga - gb) / gb


def chi_error(a, b):
    if "chi" not in a or "chi" not in b:
        return None
    return np.abs(a["chi"] - b["chi"]) / np.maximum(np.abs(b["chi"]), CHI_FLOOR)


def two_sample_chi2(a, b, edges):
    """Two-sample chi2 of the histograms of a and b on the given bin edges
    (values outside fall in the end bins); returns (statistic, dof, p).
    Bins empty in both samples are left out; the totals may differ."""
    a = np.clip(np.asarray(a, float), edges[0], edges[-1])
    b = np.clip(np.asarray(b, float), edges[0], edges[-1])
    ha = np.histogram(a, bins=edges)[0].astype(float)
    hb = np.histogram(b, bins=edges)[0].astype(float)
    keep = (ha + hb) > 0
    ha, hb = ha[keep], hb[keep]
    na, nb = ha.sum(), hb.sum()
    if na == 0 or nb == 0:
        return 0.0, 0, 1.0
    ka, kb = np.sqrt(nb / na), np.sqrt(na / nb)
    stat = float(np.sum((ka * ha - kb * hb) ** 2 / (ha + hb)))
    dof = int(keep.sum()) - 1
    import scipy.stats as st
    return stat, dof, float(st.chi2.sf(stat, max(dof, 1)))


def distribution_check(gpu, ora, label, p_min=1e-3, nbins=20):
    """Whole-population comparison by chi2 (the spectra and event-count
    distributions of the run, every particle included): final energies on
    bins equiprobable under the oracle, and per-particle emission counts.
    Returns the report; asserts p > p_min for each."""
    rep = {}
    ga = np.sqrt(1.0 + gpu["ux"] ** 2 + gpu["uy"] ** 2 + gpu["uz"] ** 2)
    gb = np.sqrt(1.0 + ora["ux"] ** 2 + ora["uy"] ** 2 + ora["uz"] ** 2)
    if len(gb) >= 10 * nbins:
        edges = np.unique(np.quantile(gb, np.linspace(0.0, 1.0, nbins + 1)))
        if len(edges) >= 3:
            rep["energy"] = two_sample_chi2(ga, gb, edges)
    if "nemit" in gpu and "nemit" in ora and len(ora["nemit"]):
        top = int(max(gpu["nemit"].max(), ora["nemit"].max()))
        if top > 0:
            # integer counts, the sparse tail pooled into its last bin
            cnt = np.bincount(ora["nemit"], minlength=top + 1)
            last = top
            while last > 1 and cnt[last:].sum() < 5:
                last -= 1
            edges = np.append(np.arange(last + 1) - 0.5, top + 0.5)
            rep["nemit"] = two_sample_chi2(gpu["nemit"], ora["nemit"], edges)
    print(f"[{label}] chi2 " + " ".join(f"{k}: stat={v[0]:.3g} dof={v[1]} p={v[2]:.3g}"
                                        for k, v in rep.items()))
    for k, v in rep.items():
        assert v[2] > p_min, (label, k, v)
    return rep


def momentum_error(a, b):
    """Per particle: max over components of |a - b| / max(|u_b|, 1)."""
    umag = np.maximum(np.sqrt(b["ux"] ** 2 + b["uy"] ** 2 + b["uz"] ** 2), 1.0)
    return np.max([np.abs(a[c] - b[c]) / umag for c in ("ux", "uy", "uz")], axis=0)


def position_error(a, b):
    return np.max([np.abs(a[c] - b[c]) / np.maximum(np.abs(b[c]), 1.0)
                   for c in ("x", "y", "z") if b.get(c) is not None], axis=0)


def head(d, n, idx=None):
    """First n entries of every array of d (or the entries idx)."""
    if idx is not None:
        return {k: (None if v is None else v[idx]) for k, v in d.items()}
    return {k: (None if v is None else v[:n]) for k, v in d.items()}


def chaos_aware_compare(gpu, ora, twin, rtol, label, margin=None, margin_min=0.0,
                        min_comparable=0.5):
    """Compare per particle where the comparison is meaningful.

    A particle is comparable when its twin oracle run (momenta kicked at the
    rounding level of the path under test after every step) stays within
    rtol/10 of the oracle, and, with `margin`, when none of its optical-depth
    decisions was closer than margin_min.  Comparable particles must have
    identical event counts and meet rtol in momentum, energy, position and
    chi; the others are counted and reported.  `twin` may be a list of twin runs with independent
    kick patterns (one twin can end close to the oracle by chance, e.g. when
    a particle leaves the pulse with a small difference of large momenta);
    the largest twin error counts.  Returns the report."""
    n = len(ora["x"])
    eu = momentum_error(gpu, ora)
    ex = position_error(gpu, ora)
    twins = twin if isinstance(twin, (list, tuple)) else [twin]
    et = np.max([np.maximum(momentum_error(t, ora), position_error(t, ora)) for t in twins],
                axis=0)
    comparable = et <= rtol / 10.0
    if margin is not None:
        comparable &= margin >= margin_min
    same_events = np.ones(n, bool)
    if "nemit" in gpu and "nemit" in ora:
        same_events = gpu["nemit"] == ora["nemit"]
    c = comparable
    eg = gamma_error(gpu, ora)
    report = {
        "particles": n, "comparable": int(c.sum()),
        "u_q99": float(np.quantile(eu[c], 0.99)) if c.any() else 0.0,
        "u_max": float(eu[c].max()) if c.any() else 0.0,
        "u_median": float(np.median(eu[c])) if c.any() else 0.0,
        "gamma_max": float(eg[c].max()) if c.any() else 0.0,
        "x_max": float(ex[c].max()) if c.any() else 0.0,
        "events_equal_comparable": int((same_events & c).sum()),
        "events_equal_all": int(same_events.sum()),
        "u_median_all": float(np.median(eu)),
    }
    report.update(chi_report(gpu, ora, c))
    print(f"\n[{label}] " + " ".join(f"{k}={v:.3g}" if isinstance(v, float) else f"{k}={v}"
                                  for k, v in report.items()))
    assert c.mean() >= min_comparable, report
    # every comparable particle meets the bar (the strict per-step gate is
    # the teacher-forced test), with identical per-particle event counts;
    # the median over every particle meets it too
    assert report["u_max"] <= rtol, report
    assert report["gamma_max"] <= rtol, report
    assert report["x_max"] <= rtol, report
    if "chi_median" in report:
        assert report["chi_median"] <= rtol and report["chi_abs_over_max"] <= rtol, report
    assert report["events_equal_comparable"] == report["comparable"], report
    assert report["u_median_all"] <= rtol, report
    return report


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
    if "nemit" in gpu and "nemit" in ora:
        assert np.array_equal(gpu["nemit"], ora["nemit"]), f"{label}: per-particle events differ"
    e = np.abs(gpu["tau"] - ora["tau"]) / np.maximum(np.abs(ora["tau"]), 1.0)
    assert e.max() <= rtol, f"{label} tau: max err {e.max():.3g} at slot {e.argmax()}"
    np.testing.assert_array_equal(gpu["w"], ora["w"])
    return worst


def teacher_forced_compare(before, gpu_after, ora_sp, rtol, margin_min, label):
    """One step from the same state on both sides.  Per species: slots that
    existed before the step are compared one by one (momentum, position,
    optical depth, per-particle event count), skipping particles whose
    optical-depth or regime decision in the oracle had a relative margin
    below margin_min; the particles appended during the step are compared
    slot by slot when every decision agreed (the appended order is then the
    same), else only their number is reported.  Returns a report per species."""
    reports = {}
    for name in SPECIES:
        b = before[name]
        g = gpu_after[name]
        o = oracle_arrays(ora_sp[name])
        n0 = len(b["x"])
        n_g, n_o = len(g["x"]), len(o["x"])
        marg = ora_sp[name].margin[:n0] if ora_sp[name].margin is not None else np.ones(n0)
        ok = marg >= margin_min
        r = {"before": n0, "after_gpu": n_g, "after_oracle": n_o, "marginal": int((~ok).sum())}
        if n0:
            gh, oh = head(g, n0), head(o, n0)
            eu = momentum_error(gh, oh)
            ex = position_error(gh, oh)
            et = np.abs(gh["tau"] - oh["tau"]) / np.maximum(np.abs(oh["tau"]), 1.0)
            eg = gamma_error(gh, oh)
            r.update(u_max=float(eu[ok].max()) if ok.any() else 0.0,
                     u_median=float(np.median(eu[ok])) if ok.any() else 0.0,
                     gamma_max=float(eg[ok].max()) if ok.any() else 0.0,
                     x_max=float(ex[ok].max()) if ok.any() else 0.0,
                     tau_max=float(et[ok].max()) if ok.any() else 0.0)
            if name != "photon":
                r.update(chi_report(gh, oh, ok))
            if "nemit" in g and "nemit" in b and ora_sp[name].nemit is not None:
                d_g = gh["nemit"] - b["nemit"]
                same = d_g == oh["nemit"]
                r["events_differ"] = int((~same & ok).sum())
                r["events_differ_marginal"] = int((~same & ~ok).sum())
                assert r["events_differ"] == 0, (label, name, r)
            dead_g, dead_o = gh["tau"] < 0, oh["tau"] < 0
            if name == "photon":
                assert np.array_equal(dead_g[ok], dead_o[ok]), (label, name, "dead photons differ")
            assert r["u_max"] <= rtol and r["x_max"] <= rtol and r["tau_max"] <= rtol, (label, name, r)
            assert r["gamma_max"] <= rtol, (label, name, r)
            assert r.get("chi_median", 0.0) <= rtol and r.get("chi_abs_over_max", 0.0) <= rtol, \
                (label, name, r)
        if r["marginal"] == 0 and n_g == n_o and n_g > n0:
            ga, oa = head({k: v[n0:] for k, v in g.items() if v is not None}, n_g - n0), \
                head({k: v[n0:] for k, v in o.items() if v is not None}, n_o - n0)
            ea = momentum_error(ga, oa)
            r["appended_u_max"] = float(ea.max())
            assert r["appended_u_max"] <= rtol, (label, name, r)
        reports[name] = r
    print(f"\n[{label}] " + "; ".join(
        f"{k}: " + " ".join(f"{a}={v:.3g}" if isinstance(v, float) else f"{a}={v}"
                            for a, v in r.items()) for k, r in reports.items()))
    return reports
