"""ctypes binding of libqedpic (include/qedpic.h), same names as the C ABI.

Argument marshalling only: every step of the QED particle path runs in the
library's CUDA kernels.  Importing this module does not load the library;
the first call does, and raises if ``libqedpic.so`` has not been built (there
is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

QP_OK = 0
QP_WARN_BUFFER_FULL = 1
QP_WARN_TABLE_CLAMPED = 2
QP_ERR_INVALID_ARG = -1
QP_ERR_CUDA = -2
QP_ERR_OOM = -3
QP_ERR_NOT_INITIALIZED = -4
QP_ERR_TIMEOUT = -5

QP_ELECTRON, QP_POSITRON, QP_PHOTON = 0, 1, 2
QP_FP64, QP_MIXED = 0, 1
QP_FIELD_NONE, QP_FIELD_PLANE, QP_FIELD_GAUSSIAN, QP_FIELD_YEE2D, QP_FIELD_UNIFORM_B = range(5)
QP_MAX_EMISSIONS = 8
QP_MAX_BATCH = 64
QP_STEP_TILE = 128
QP_HIST_BINS = 64
QP_NRATE, QP_NCDF, QP_NNODE = 769, 97, 256

FIELD_KINDS = {"none": QP_FIELD_NONE, "plane": QP_FIELD_PLANE, "gaussian": QP_FIELD_GAUSSIAN,
               "yee2d": QP_FIELD_YEE2D, "uniform_b": QP_FIELD_UNIFORM_B}

_dp = C.POINTER(C.c_double)


class qp_table_params(C.Structure):
    _fields_ = [("lambda_m", C.c_double), ("device", C.c_int32), ("reserved", C.c_int32)]


class qp_species_desc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("dims", C.c_int32), ("capacity", C.c_int64),
                ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p),
                ("ux", C.c_void_p), ("uy", C.c_void_p), ("uz", C.c_void_p),
                ("tau", C.c_void_p), ("w", C.c_void_p), ("chi", C.c_void_p),
                ("nemit", C.c_void_p), ("n_live", C.c_void_p), ("id_base", C.c_int64),
                ("id_split", C.c_int64), ("id_append", C.c_int64)]


class qp_field(C.Structure):
    _fields_ = [("kind", C.c_int32), ("reserved", C.c_int32), ("a0", C.c_double),
                ("w0", C.c_double), ("tau_fwhm", C.c_double), ("x_focus", C.c_double),
                ("t_focus", C.c_double), ("b0", C.c_double), ("yee", C.c_void_p * 6),
                ("nx", C.c_int64), ("ny", C.c_int64), ("dx", C.c_double), ("dy", C.c_double),
                ("x0", C.c_double), ("y0", C.c_double)]


class qp_step_params(C.Structure):
    _fields_ = [("field", qp_field), ("dt", C.c_double), ("step", C.c_int64),
                ("n_steps", C.c_int32), ("precision", C.c_int32), ("seed", C.c_uint64),
                ("chi_threshold", C.c_double), ("photon_min_gamma", C.c_double),
                ("pairs", C.c_int32), ("max_emissions", C.c_int32), ("electron", C.c_int32),
                ("positron", C.c_int32), ("photon", C.c_int32), ("reserved", C.c_int32)]


class qp_host_state(C.Structure):
    _fields_ = [("host", C.c_void_p), ("pitch", C.c_int64), ("count", C.c_int64)]


class qp_diag(C.Structure):
    _fields_ = ([("n_live", C.c_int64), ("n_alive", C.c_int64)]
                + [(n, C.c_double) for n in ("weight", "energy", "px", "py", "pz", "chi_mean")]
                + [("hist", C.c_double * QP_HIST_BINS)]
                + [(n, C.c_int64) for n in ("n_emit", "n_photon", "n_photon_drop",
                                            "n_subthreshold", "n_pair", "n_pair_drop",
                                            "n_saturated", "n_clamped", "n_continuous")]
                + [("e_subthreshold", C.c_double), ("e_dropped", C.c_double),
                   ("status", C.c_int32), ("reserved", C.c_int32)])

    def as_dict(self):
        d = {n: getattr(self, n) for n, _ in self._fields_ if n not in ("hist", "reserved")}
        d["hist"] = list(self.hist)
        return d


class qp_tables_export(C.Structure):
    _fields_ = [("H", C.c_double * QP_NRATE), ("Gs", C.c_double * QP_NRATE),
                ("Ts", C.c_double * QP_NRATE), ("Cg", C.c_double * (QP_NCDF * QP_NNODE)),
                ("Cp", C.c_double * (QP_NCDF * QP_NNODE)), ("a_S", C.c_double),
                ("C_rate", C.c_double), ("tau0w", C.c_double)]


class QPError(RuntimeError):
    def __init__(self, fn, status):
        super().__init__(f"{fn} returned {status_name(status)} ({status})")
        self.status = status


_lock = threading.Lock()
_lib = None

class qp_pulse2d(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("a0", "w0", "tau_fwhm", "x_focus", "t_focus",
                                          "y_axis")]


class qp_coalesce_params(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("x0", "y0", "z0", "dx", "dy", "dz")] + [
        ("nx", C.c_int64), ("ny", C.c_int64), ("nz", C.c_int64),
        ("energy_bins_per_octave", C.c_int32), ("direction_bins", C.c_int32),
        ("min_group", C.c_int32), ("max_group", C.c_int32), ("seed", C.c_uint64),
        ("step", C.c_int64)]


class qp_coalesce_stats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("groups_merged", "photons_merged", "n_before",
                                         "n_after")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


EXPORTS = ("qp_init_tables", "qp_destroy", "qp_create_species", "qp_init_optical_depth",
           "qp_species_copy", "qp_step_host",
           "qp_step", "qp_diagnostics", "qp_export_tables", "qp_reset_counters",
           "qp_selftest_wait_timeout", "qp_profile_enable", "qp_profile_read",
           "qp_diagnostics_noalloc", "qp_status_string", "qp_destroy_species",
           "qp_batch_create", "qp_batch_destroy", "qp_batch_scratch_words", "qp_batch_set",
           "qp_batch_clear", "qp_batch_step", "qp_batch_progress", "qp_coalesce_photons",
           "qp_compact_photons", "qp_fill_yee2d", "qp_step_fused", "qp_yee_advance_b",
           "qp_yee_advance_e", "qp_deposit_current", "qp_sort_species")


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = False):
    """The loaded libqedpic (raises if it is not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"{path} is missing: build it with "
                                   "`python -m paper_1311_1107_gb300.build` (no CPU fallback)")
            _build.build()
        L = C.CDLL(path)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        L.qp_init_tables.argtypes = [C.POINTER(qp_table_params), C.POINTER(vp)]
        L.qp_destroy.argtypes = [vp]
        L.qp_create_species.argtypes = [vp, C.POINTER(qp_species_desc), C.POINTER(i32)]
        L.qp_init_optical_depth.argtypes = [vp, i32, C.c_uint64, i64, i64, vp]
        L.qp_species_copy.argtypes = [vp, i32, vp, i64, i64, i32, vp]
        L.qp_step_host.argtypes = [vp, C.POINTER(qp_step_params), C.POINTER(qp_host_state), vp]
        L.qp_step.argtypes = [vp, C.POINTER(qp_step_params), vp]
        L.qp_diagnostics.argtypes = [vp, i32, C.POINTER(qp_diag), vp]
        L.qp_diagnostics_noalloc.argtypes = [C.POINTER(qp_species_desc), C.POINTER(qp_diag), vp]
        L.qp_export_tables.argtypes = [vp, C.POINTER(qp_tables_export)]
        L.qp_reset_counters.argtypes = [vp, i32]
        L.qp_selftest_wait_timeout.argtypes = [vp, C.c_uint32]
        L.qp_profile_enable.argtypes = [vp, C.c_int]
        L.qp_profile_read.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
        L.qp_destroy_species.argtypes = [vp, i32]
        L.qp_batch_create.argtypes = [vp, i32, i32, i32, C.POINTER(vp)]
        L.qp_batch_destroy.argtypes = [vp]
        L.qp_batch_scratch_words.argtypes = [vp, C.POINTER(qp_step_params), C.POINTER(i64)]
        L.qp_batch_set.argtypes = [vp, i32, C.POINTER(qp_step_params), vp, i64, vp]
        L.qp_batch_clear.argtypes = [vp, i32, vp]
        L.qp_batch_step.argtypes = [vp, i32, vp]
        L.qp_batch_progress.argtypes = [vp, vp, vp, vp, vp]
        L.qp_status_string.argtypes = [C.c_int]
        L.qp_coalesce_photons.argtypes = [vp, i32, C.POINTER(qp_coalesce_params),
                                          C.POINTER(qp_coalesce_stats), vp]
        L.qp_compact_photons.argtypes = [vp, i32, C.POINTER(qp_coalesce_stats), vp]
        L.qp_step_fused.argtypes = [vp, C.POINTER(qp_step_params), i32, vp]
        L.qp_yee_advance_b.argtypes = [vp, C.POINTER(qp_field), C.c_double, vp]
        L.qp_yee_advance_e.argtypes = [vp, C.POINTER(qp_field), vp, vp, vp, C.c_double, vp]
        L.qp_deposit_current.argtypes = [vp, i32, C.POINTER(qp_field), vp, vp, vp, C.c_double,
                                         vp]
        L.qp_sort_species.argtypes = [vp, i32, C.POINTER(qp_field), vp]
        L.qp_fill_yee2d.argtypes = [vp, C.POINTER(qp_pulse2d), C.POINTER(qp_field), C.c_double,
                                    vp]
        L.qp_status_string.restype = C.c_char_p
        for name in EXPORTS:
            if name != "qp_status_string":
                getattr(L, name).restype = C.c_int
        _lib = L
        return L


def status_name(status: int) -> str:
    return lib().qp_status_string(int(status)).decode()


def _check(fn, st, allow_warn=True):
    if st < 0 or (st > 0 and not allow_warn):
        raise QPError(fn, st)
    return st


# ---------------------------------------------------------------- the C calls

def qp_init_tables(lambda_m: float = 0.8e-6, device: int = 0) -> C.c_void_p:
    p = qp_table_params(lambda_m, device, 0)
    ctx = C.c_void_p()
    _check("qp_init_tables", lib().qp_init_tables(C.byref(p), C.byref(ctx)))
    return ctx


def qp_destroy(ctx) -> int:
    return lib().qp_destroy(ctx)


def qp_create_species(ctx, desc: qp_species_desc) -> int:
    h = C.c_int32(-1)
    _check("qp_create_species", lib().qp_create_species(ctx, C.byref(desc), C.byref(h)))
    return h.value


def qp_init_optical_depth(ctx, handle: int, seed: int, first: int, count: int, stream=None):
    return _check("qp_init_optical_depth",
                  lib().qp_init_optical_depth(ctx, handle, seed, first, count, stream))


def qp_species_copy(ctx, handle: int, host_ptr: int, host_pitch: int, count: int,
                    to_device: bool, stream=None):
    """Slots [0, count) of the FP64 state between the device arrays and a host
    block (array k at host_ptr + k * host_pitch bytes)."""
    return _check("qp_species_copy",
                  lib().qp_species_copy(ctx, handle, host_ptr, host_pitch, count,
                                        1 if to_device else 0, stream))


def qp_step_host(ctx, params: qp_step_params, states, stream=None) -> int:
    """params.n_steps steps of state held in host blocks: states is a
    qp_host_state[3] array (electron, positron, photon); their counts are
    updated to the live counts after the steps."""
    return _check("qp_step_host", lib().qp_step_host(ctx, C.byref(params), states, stream))


def qp_step(ctx, params: qp_step_params, stream=None) -> int:
    return _check("qp_step", lib().qp_step(ctx, C.byref(params), stream))


def qp_diagnostics(ctx, handle: int, stream=None) -> qp_diag:
    d = qp_diag()
    st = lib().qp_diagnostics(ctx, handle, C.byref(d), stream)
    if st < 0 and d.status != st:
        raise QPError("qp_diagnostics", st)
    return d


def qp_diagnostics_noalloc(desc: qp_species_desc, stream=None) -> qp_diag:
    """Allocation-free reduction of one species (no context; see the header:
    a static scratch array limits the species to QP_NOALLOC_MAX_SLOTS)."""
    d = qp_diag()
    _check("qp_diagnostics_noalloc", lib().qp_diagnostics_noalloc(C.byref(desc), C.byref(d), stream))
    return d


QP_NOALLOC_MAX_SLOTS = 4096 * 256


def qp_export_tables(ctx) -> qp_tables_export:
    t = qp_tables_export()
    _check("qp_export_tables", lib().qp_export_tables(ctx, C.byref(t)))
    return t


def qp_reset_counters(ctx, handle: int) -> int:
    return _check("qp_reset_counters", lib().qp_reset_counters(ctx, handle))


def qp_selftest_wait_timeout(ctx, spin_limit: int) -> int:
    """Status raised by a deliberately unsatisfiable, bounded device wait."""
    return lib().qp_selftest_wait_timeout(ctx, int(spin_limit))


def qp_profile_enable(ctx, enable: bool = True) -> int:
    return _check("qp_profile_enable", lib().qp_profile_enable(ctx, 1 if enable else 0))


def qp_profile_read(ctx):
    """(ms[3], launches[3]): entry 0 is the fused step kernel; 1 and 2 are reserved (0)."""
    ms = (C.c_double * 3)()
    n = (C.c_int64 * 3)()
    _check("qp_profile_read", lib().qp_profile_read(ctx, ms, n))
    return list(ms), list(n)


def qp_status_string(status: int) -> str:
    return status_name(status)


def qp_destroy_species(ctx, handle: int) -> int:
    return _check("qp_destroy_species", lib().qp_destroy_species(ctx, int(handle)))


# ---------------------------------------------------------------- batches

def qp_batch_create(ctx, max_problems: int, precision: int, field_kind: int) -> C.c_void_p:
    b = C.c_void_p()
    _check("qp_batch_create", lib().qp_batch_create(ctx, int(max_problems), int(precision),
                                                    int(field_kind), C.byref(b)))
    return b


def qp_batch_destroy(batch) -> int:
    return _check("qp_batch_destroy", lib().qp_batch_destroy(batch))


def qp_batch_scratch_words(ctx, params: qp_step_params) -> int:
    w = C.c_int64(0)
    _check("qp_batch_scratch_words", lib().qp_batch_scratch_words(ctx, C.byref(params),
                                                                  C.byref(w)))
    return w.value


def qp_batch_set(batch, slot: int, params: qp_step_params, scratch_ptr: int, scratch_words: int,
                 stream=None) -> int:
    return _check("qp_batch_set", lib().qp_batch_set(batch, int(slot), C.byref(params),
                                                     C.c_void_p(scratch_ptr),
                                                     int(scratch_words), stream))


def qp_batch_clear(batch, slot: int, stream=None) -> int:
    return _check("qp_batch_clear", lib().qp_batch_clear(batch, int(slot), stream))


def qp_batch_step(batch, n_launches: int, stream=None) -> int:
    return _check("qp_batch_step", lib().qp_batch_step(batch, int(n_launches), stream))


def qp_batch_progress(batch, steps_left_ptr: int, next_step_ptr: int | None = None,
                      work_ptr: int | None = None, stream=None) -> int:
    """Enqueue copies of the slots' remaining launches (and next steps, and
    live slots stepped) into host memory at the given addresses (pinned,
    max_problems int64 each)."""
    opt = lambda p: None if p is None else C.c_void_p(p)
    return _check("qp_batch_progress", lib().qp_batch_progress(
        batch, C.c_void_p(steps_left_ptr), opt(next_step_ptr), opt(work_ptr), stream))


def coalesce_params(box, cells, energy_bins_per_octave=8, direction_bins=8, min_group=3,
                    seed=0, step=0, max_group=0) -> qp_coalesce_params:
    """box: (x0, y0, z0, dx, dy, dz); cells: (nx, ny, nz); max_group 0: 256."""
    p = qp_coalesce_params()
    p.x0, p.y0, p.z0, p.dx, p.dy, p.dz = (float(v) for v in box)
    p.nx, p.ny, p.nz = (int(v) for v in cells)
    p.energy_bins_per_octave, p.direction_bins = energy_bins_per_octave, direction_bins
    p.min_group, p.seed, p.step = min_group, seed, step
    p.max_group = max_group
    return p


def qp_coalesce_photons(ctx, handle: int, params: qp_coalesce_params | None, stream=None,
                        stats: bool = True):
    """Compaction (params None) or coalescence of a photon species; with
    stats, synchronises the stream and returns the counts as a dict."""
    out = qp_coalesce_stats() if stats else None
    _check("qp_coalesce_photons",
           lib().qp_coalesce_photons(ctx, handle, None if params is None else C.byref(params),
                                     None if out is None else C.byref(out), stream))
    return out.as_dict() if out is not None else None


def qp_compact_photons(ctx, handle: int, stream=None, stats: bool = True):
    out = qp_coalesce_stats() if stats else None
    _check("qp_compact_photons",
           lib().qp_compact_photons(ctx, handle, None if out is None else C.byref(out), stream))
    return out.as_dict() if out is not None else None


def pulse2d(a0, w0, tau_fwhm, x_focus, t_focus, y_axis) -> qp_pulse2d:
    p = qp_pulse2d()
    p.a0, p.w0, p.tau_fwhm, p.x_focus, p.t_focus, p.y_axis = (float(v) for v in (
        a0, w0, tau_fwhm, x_focus, t_focus, y_axis))
    return p


def qp_fill_yee2d(ctx, pulse: qp_pulse2d, grid: qp_field, t: float, stream=None) -> int:
    return _check("qp_fill_yee2d",
                  lib().qp_fill_yee2d(ctx, C.byref(pulse), C.byref(grid), float(t), stream))


def qp_step_fused(ctx, params: qp_step_params, fuse: int, stream=None) -> int:
    """params.n_steps steps, `fuse` per launch window (pairs off; the same
    results as qp_step)."""
    return _check("qp_step_fused", lib().qp_step_fused(ctx, C.byref(params), int(fuse), stream))


def qp_yee_advance_b(ctx, grid: qp_field, dtb: float, stream=None) -> int:
    return _check("qp_yee_advance_b", lib().qp_yee_advance_b(ctx, C.byref(grid), float(dtb),
                                                             stream))


def qp_yee_advance_e(ctx, grid: qp_field, jx_ptr, jy_ptr, jz_ptr, dt: float, stream=None) -> int:
    """j*_ptr: device addresses (int) of the current arrays, or None."""
    return _check("qp_yee_advance_e", lib().qp_yee_advance_e(ctx, C.byref(grid), jx_ptr, jy_ptr,
                                                             jz_ptr, float(dt), stream))


def qp_deposit_current(ctx, handle: int, grid: qp_field, jx_ptr, jy_ptr, jz_ptr, dt: float,
                       stream=None) -> int:
    return _check("qp_deposit_current",
                  lib().qp_deposit_current(ctx, handle, C.byref(grid), jx_ptr, jy_ptr, jz_ptr,
                                           float(dt), stream))


def qp_sort_species(ctx, handle: int, grid: qp_field, stream=None) -> int:
    return _check("qp_sort_species", lib().qp_sort_species(ctx, handle, C.byref(grid), stream))
