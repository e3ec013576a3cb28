"""FP64 CPU oracle of the QED particle step (test infrastructure only).

This package is the plain, slow reference the CUDA library is checked against.
It is written from the paper (Lobet et al., arXiv:1311.1107, sections 2-3:
Eq. 1-8 and the Monte-Carlo pair scheme) and shares no code with the library.
Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the product path never does.

The arithmetic lives in ``qed_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off`` so that results do not depend on the host's FMA
contraction).  This module compiles it with gcc on first use and exposes it
through ctypes with numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qed_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# grid sizes of the table definition (see qed_oracle.c)
NRATE, NCDF, NS = 769, 97, 256

ELECTRON, POSITRON, PHOTON = 0, 1, 2
RNG_INIT, RNG_EMIT, RNG_PHOTON_TAU, RNG_PAIR, RNG_PAIR_POS = 0, 1, 2, 3, 4
FIELD_NONE, FIELD_PLANE, FIELD_GAUSSIAN, FIELD_YEE2D, FIELD_UNIFORM_B = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, FP64, no FMA contraction)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


class Units(C.Structure):
    _fields_ = [("lambda_m", C.c_double), ("omega", C.c_double), ("tau_c", C.c_double),
                ("a_S", C.c_double), ("C_rate", C.c_double), ("tau0w", C.c_double),
                ("alpha", C.c_double)]


class Field(C.Structure):
    _fields_ = [("kind", C.c_int), ("a0", C.c_double), ("w0", C.c_double),
                ("tau_fwhm", C.c_double), ("x_focus", C.c_double), ("t_focus", C.c_double),
                ("b0", C.c_double), ("yee", C.c_void_p * 6), ("nx", C.c_int64),
                ("ny", C.c_int64), ("dx", C.c_double), ("dy", C.c_double),
                ("x0", C.c_double), ("y0", C.c_double)]


class _Species(C.Structure):
    _fields_ = [("n", C.c_int64), ("cap", C.c_int64)] + [
        (name, C.c_void_p) for name in ("x", "y", "z", "ux", "uy", "uz", "tau", "w", "chi",
                                        "margin", "nemit", "ids")] + [
        ("id_base", C.c_int64), ("id_split", C.c_int64), ("id_append", C.c_int64)]


class Params(C.Structure):
    _fields_ = [("dt", C.c_double), ("step", C.c_int64), ("seed", C.c_uint64),
                ("chi_th", C.c_double), ("photon_min_gamma", C.c_double),
                ("pairs", C.c_int32), ("max_emit", C.c_int32), ("recoil", C.c_int32),
                ("dims", C.c_int32), ("noise", C.c_double), ("noise_key", C.c_uint64)]


class CoalesceParams(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("x0", "y0", "z0", "dx", "dy", "dz")] + [
        ("nx", C.c_int64), ("ny", C.c_int64), ("nz", C.c_int64),
        ("ebins_per_octave", C.c_int32), ("dir_bins", C.c_int32), ("min_group", C.c_int32),
        ("dims", C.c_int32), ("max_group", C.c_int32), ("pad", C.c_int32),
        ("seed", C.c_uint64), ("step", C.c_int64)]


class CoalesceStats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("n_before", "n_dead", "n_after", "groups_merged",
                                         "photons_merged")]


class Pulse2D(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("a0", "w0", "tau_fwhm", "x_focus", "t_focus",
                                          "y_axis")]


class Stats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("n_emit", "n_photon", "n_photon_drop",
                                         "n_subthreshold", "n_pair", "n_pair_drop",
                                         "n_saturated", "n_clamped", "n_continuous")] + [
        ("e_subthreshold", C.c_double), ("e_dropped", C.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        d, i64, u32p = C.c_double, C.c_int64, C.POINTER(C.c_uint32)
        vp = C.c_void_p
        sig = {
            "or_units_init": (None, [d, C.POINTER(Units)]),
            "or_bessel_K": (d, [d, d]),
            "or_int_K13": (d, [d]),
            "or_F_gamma": (d, [d, d, d]),
            "or_F_pair": (d, [d, d, d]),
            "or_H_exact": (d, [d]),
            "or_G_exact": (d, [d]),
            "or_T_exact": (d, [d]),
            "or_cdf_gamma_exact": (d, [d, d]),
            "or_cdf_pair_exact": (d, [d, d]),
            "or_tables_size": (C.c_size_t, []),
            "or_tables_build": (None, [vp]),
            "or_lookup_rate": (d, [vp, C.c_int, d, C.POINTER(C.c_int)]),
            "or_sample_gamma": (d, [vp, d, d, C.POINTER(C.c_int)]),
            "or_sample_pair": (d, [vp, d, d, C.POINTER(C.c_int)]),
            "or_philox4x32_10": (None, [u32p, u32p, u32p]),
            "or_u53": (d, [C.c_uint32, C.c_uint32]),
            "or_draw": (None, [C.c_uint64, C.c_int, C.c_int, i64, i64, C.c_int, u32p]),
            "or_field_eval": (None, [C.POINTER(Field), d, d, d, d, vp, vp]),
            "or_chi_e": (d, [vp, vp, vp, d, d]),
            "or_chi_gamma": (d, [vp, vp, vp, d]),
            "or_boris": (None, [d, d, vp, vp, vp]),
            "or_step": (C.c_int, [C.POINTER(Units), vp, C.POINTER(Field), C.POINTER(Params),
                                  C.POINTER(_Species), C.POINTER(_Species),
                                  C.POINTER(_Species), C.POINTER(Stats)]),
            "or_run": (C.c_int, [C.POINTER(Units), vp, C.POINTER(Field), C.POINTER(Params),
                                 i64, C.POINTER(_Species), C.POINTER(_Species),
                                 C.POINTER(_Species), C.POINTER(Stats)]),
            "or_init_tau": (None, [C.c_uint64, C.c_int, vp, i64, i64]),
            "or_coalesce": (C.c_int, [C.POINTER(_Species), C.POINTER(CoalesceParams),
                                      C.POINTER(CoalesceStats)]),
            "or_pulse2d_eval": (d, [C.POINTER(Pulse2D), d, d, d]),
            "or_yee_advance_b": (None, [C.POINTER(vp), i64, i64, d, d, d]),
            "or_yee_advance_e": (None, [C.POINTER(vp), C.POINTER(vp), i64, i64, d, d, d]),
            "or_deposit_current": (None, [C.POINTER(_Species), d, d, C.POINTER(vp), i64, i64, d,
                                          d, d, d]),
            "or_sort_by_cell": (C.c_int, [C.POINTER(_Species), i64, i64, d, d, d, d]),
            "or_fill_pulse2d": (None, [C.POINTER(Pulse2D), vp, vp, i64, i64, d, d, d, d, d]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _vec(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(3))


# ---------------------------------------------------------------- units, functions

def units(lambda_m: float = 0.8e-6) -> Units:
    u = Units()
    lib().or_units_init(lambda_m, C.byref(u))
    return u


def bessel_K(nu, x):
    f = lib().or_bessel_K
    return np.vectorize(lambda xx: f(float(nu), float(xx)), otypes=[float])(x)


def int_K13(x):
    f = lib().or_int_K13
    return np.vectorize(lambda xx: f(float(xx)), otypes=[float])(x)


def F_gamma(u, chi, omu=None):
    """Eq. 2 bracket (positive reading) at photon fraction u."""
    f = lib().or_F_gamma
    u = np.asarray(u, dtype=float)
    omu = 1.0 - u if omu is None else np.asarray(omu, dtype=float)
    return np.vectorize(lambda a, b: f(float(a), float(b), float(chi)), otypes=[float])(u, omu)


def F_pair(v, chi, omv=None):
    f = lib().or_F_pair
    v = np.asarray(v, dtype=float)
    omv = 1.0 - v if omv is None else np.asarray(omv, dtype=float)
    return np.vectorize(lambda a, b: f(float(a), float(b), float(chi)), otypes=[float])(v, omv)


def H_exact(chi):
    return np.vectorize(lambda c: lib().or_H_exact(float(c)), otypes=[float])(chi)


def G_exact(chi):
    return np.vectorize(lambda c: lib().or_G_exact(float(c)), otypes=[float])(chi)


def T_exact(chi):
    return np.vectorize(lambda c: lib().or_T_exact(float(c)), otypes=[float])(chi)


def cdf_gamma_exact(s, chi):
    """Eq. 7 CDF at the photon fraction with logit s."""
    return np.vectorize(lambda a: lib().or_cdf_gamma_exact(float(a), float(chi)),
                        otypes=[float])(s)


def cdf_pair_exact(s, chi):
    return np.vectorize(lambda a: lib().or_cdf_pair_exact(float(a), float(chi)),
                        otypes=[float])(s)


# ---------------------------------------------------------------- tables

class Tables:
    """The oracle's own rate and CDF tables (built from its own quadrature)."""

    def __init__(self):
        n = lib().or_tables_size()
        self._buf = np.zeros(n // 8, dtype=np.float64)
        lib().or_tables_build(self.ptr)
        b = self._buf
        off = 0

        def take(k):
            nonlocal off
            a = b[off:off + k]
            off += k
            return a
        self.chi, self.H, self.Gs, self.Ts = take(NRATE), take(NRATE), take(NRATE), take(NRATE)
        self.chic = take(NCDF)
        self.sg, self.ug, self.sp, self.vp = take(NS), take(NS), take(NS), take(NS)
        self.Cg = take(NCDF * NS).reshape(NCDF, NS)
        self.Cp = take(NCDF * NS).reshape(NCDF, NS)
        assert off * 8 == n

    @property
    def ptr(self):
        return self._buf.ctypes.data_as(C.c_void_p)

    def lookup(self, which: int, chi: float):
        cl = C.c_int(0)
        v = lib().or_lookup_rate(self.ptr, which, float(chi), C.byref(cl))
        return v, bool(cl.value)

    def sample_gamma(self, chi: float, xi: float) -> float:
        cl = C.c_int(0)
        return lib().or_sample_gamma(self.ptr, float(chi), float(xi), C.byref(cl))

    def sample_pair(self, chi: float, xi: float) -> float:
        cl = C.c_int(0)
        return lib().or_sample_pair(self.ptr, float(chi), float(xi), C.byref(cl))


_tables_cache = None


def tables() -> Tables:
    """Process-wide oracle tables (built once, a few seconds)."""
    global _tables_cache
    if _tables_cache is None:
        _tables_cache = Tables()
    return _tables_cache


# ---------------------------------------------------------------- RNG

def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def u53(a: int, b: int) -> float:
    return lib().or_u53(a & 0xFFFFFFFF, b & 0xFFFFFFFF)


def draw(seed, species, purpose, slot, step, k=0):
    o = (C.c_uint32 * 4)()
    lib().or_draw(int(seed), int(species), int(purpose), int(slot), int(step), int(k), o)
    return [int(v) for v in o]


# ---------------------------------------------------------------- fields, push, chi

def plane_field(a0: float) -> Field:
    f = Field()
    f.kind, f.a0 = FIELD_PLANE, a0
    return f


def gaussian_field(a0, w0, tau_fwhm, x_focus, t_focus) -> Field:
    f = Field()
    f.kind, f.a0, f.w0, f.tau_fwhm = FIELD_GAUSSIAN, a0, w0, tau_fwhm
    f.x_focus, f.t_focus = x_focus, t_focus
    return f


def uniform_b_field(b0: float) -> Field:
    f = Field()
    f.kind, f.b0 = FIELD_UNIFORM_B, b0
    return f


def yee2d_field(comps, dx, dy, x0=0.0, y0=0.0) -> Field:
    """comps: 6 float32 arrays (Ex Ey Ez Bx By Bz) of shape (ny, nx)."""
    f = Field()
    f.kind = FIELD_YEE2D
    keep = [np.array(c, dtype=np.float32, copy=True, order="C") for c in comps]
    ny, nx = keep[0].shape
    for k, c in enumerate(keep):
        f.yee[k] = c.ctypes.data
    f.nx, f.ny, f.dx, f.dy, f.x0, f.y0 = nx, ny, dx, dy, x0, y0
    f._keep = keep  # keep the arrays alive
    return f


def field_eval(field: Field, x, y, z, t):
    E = np.zeros(3)
    B = np.zeros(3)
    lib().or_field_eval(C.byref(field), float(x), float(y), float(z), float(t), _ptr(E), _ptr(B))
    return E, B


def chi_e(E, B, u, gamma, a_S):
    return lib().or_chi_e(_ptr(_vec(E)), _ptr(_vec(B)), _ptr(_vec(u)), float(gamma), float(a_S))


def chi_gamma(E, B, u, a_S):
    return lib().or_chi_gamma(_ptr(_vec(E)), _ptr(_vec(B)), _ptr(_vec(u)), float(a_S))


def boris(q, dt, E, B, u):
    uu = _vec(u).copy()
    lib().or_boris(float(q), float(dt), _ptr(_vec(E)), _ptr(_vec(B)), _ptr(uu))
    return uu


# ---------------------------------------------------------------- species and runs

class Species:
    """SoA state of one species in FP64 numpy arrays with a slot capacity."""

    NAMES = ("x", "y", "z", "ux", "uy", "uz", "tau", "w")

    def __init__(self, cap: int, dims: int = 3, track: bool = True):
        self.cap, self.dims, self.n = int(cap), dims, 0
        for nm in self.NAMES:
            if nm == "z" and dims == 2:
                setattr(self, nm, None)
            else:
                setattr(self, nm, np.zeros(self.cap))
        self.chi = np.zeros(self.cap) if track else None
        self.margin = np.full(self.cap, np.inf) if track else None
        self.nemit = np.zeros(self.cap, dtype=np.int32) if track else None
        self.ids = None  # optional int64 slot numbers for the random streams
        # without ids: slot i is particle id_base + i below id_split (when
        # id_split > 0) and id_append + (i - id_split) from there on
        self.id_base, self.id_split, self.id_append = 0, 0, 0

    @classmethod
    def from_arrays(cls, arrays: dict, cap: int, dims: int = 3, track: bool = True,
                    ids=None):
        """ids: optional slot numbers (for sampled subsets of a population)."""
        n = len(arrays["x"])
        s = cls(max(cap, n), dims, track)
        for nm in cls.NAMES:
            if nm in arrays and getattr(s, nm) is not None:
                getattr(s, nm)[:n] = np.asarray(arrays[nm], dtype=np.float64)
        s.n = n
        if ids is not None:
            s.ids = np.zeros(s.cap, dtype=np.int64)
            s.ids[:n] = np.asarray(ids, dtype=np.int64)
        return s

    def _struct(self):
        st = _Species()
        st.n, st.cap = self.n, self.cap
        st.id_base, st.id_split, st.id_append = self.id_base, self.id_split, self.id_append
        for nm in self.NAMES + ("chi", "margin", "nemit", "ids"):
            a = getattr(self, nm)
            setattr(st, nm, None if a is None else a.ctypes.data)
        return st

    def live(self, nm):
        a = getattr(self, nm)
        return None if a is None else a[:self.n]


def init_tau(seed: int, species: int, sp: Species, first: int = 0, last: int | None = None):
    last = sp.n if last is None else last
    lib().or_init_tau(int(seed), int(species), sp.tau.ctypes.data_as(C.c_void_p), first, last)


class Sim:
    """A run of the oracle: units, tables, field, parameters and three species."""

    def __init__(self, field: Field, params: dict, electrons: Species | None = None,
                 positrons: Species | None = None, photons: Species | None = None,
                 lambda_m: float = 0.8e-6, table: Tables | None = None):
        self.U = units(lambda_m)
        self.T = table if table is not None else tables()
        self.field = field
        self.P = Params()
        self.P.dt = params["dt"]
        self.P.step = int(params.get("step", 0))
        self.P.seed = int(params.get("seed", 0))
        self.P.chi_th = float(params.get("chi_th", 0.0))
        self.P.photon_min_gamma = float(params.get("photon_min_gamma", 2.0))
        self.P.pairs = int(bool(params.get("pairs", False)))
        self.P.max_emit = int(params.get("max_emit", 8))
        self.P.recoil = int(params.get("recoil", 1))
        self.P.dims = int(params.get("dims", 3))
        self.P.noise = float(params.get("noise", 0.0))
        self.P.noise_key = int(params.get("noise_key", 0))
        self.sp = [electrons, positrons, photons]
        self.stats = Stats()

    def run(self, n_steps: int):
        structs = [s._struct() if s is not None else None for s in self.sp]
        ptrs = [C.byref(s) if s is not None else None for s in structs]
        lib().or_run(C.byref(self.U), self.T.ptr, C.byref(self.field), C.byref(self.P),
                     int(n_steps), ptrs[0], ptrs[1], ptrs[2], C.byref(self.stats))
        for s, st in zip(self.sp, structs):
            if s is not None:
                s.n = st.n
        self.P.step += int(n_steps)


def coalesce_params(box, cells, ebins_per_octave=8, dir_bins=8, min_group=3, dims=3, seed=0,
                    step=0, max_group=0) -> CoalesceParams:
    """box: (x0, y0, z0, dx, dy, dz); cells: (nx, ny, nz); max_group 0: 256."""
    c = CoalesceParams()
    c.x0, c.y0, c.z0, c.dx, c.dy, c.dz = (float(v) for v in box)
    c.nx, c.ny, c.nz = (int(v) for v in cells)
    c.ebins_per_octave, c.dir_bins, c.min_group = ebins_per_octave, dir_bins, min_group
    c.dims, c.seed, c.step = dims, seed, step
    c.max_group = max_group
    return c


def coalesce(sp: Species, params: CoalesceParams | None):
    """Compaction (params None: decayed photons removed, order kept) or
    coalescence of a photon species in place; returns the stats as a dict."""
    st = CoalesceStats()
    s = sp._struct()
    r = lib().or_coalesce(C.byref(s), None if params is None else C.byref(params),
                          C.byref(st))
    if r != 0:
        raise ValueError("or_coalesce: bad parameters")
    sp.n = s.n
    return {name: getattr(st, name) for name, _ in st._fields_}


def pulse2d(a0, w0, tau_fwhm, x_focus, t_focus, y_axis) -> Pulse2D:
    p = Pulse2D()
    p.a0, p.w0, p.tau_fwhm, p.x_focus, p.t_focus, p.y_axis = (float(v) for v in (
        a0, w0, tau_fwhm, x_focus, t_focus, y_axis))
    return p


def pulse2d_eval(p: Pulse2D, x, y, t):
    f = lib().or_pulse2d_eval
    return np.vectorize(lambda a, b, c: f(C.byref(p), float(a), float(b), float(c)),
                        otypes=[float])(x, y, t)


def fill_pulse2d(p: Pulse2D, field: Field, t: float):
    """Refill E_y and B_z of a yee2d_field (its float32 arrays, in place)
    with the pulse at time t."""
    ey, bz = field._keep[1], field._keep[5]
    lib().or_fill_pulse2d(C.byref(p), ey.ctypes.data_as(C.c_void_p),
                          bz.ctypes.data_as(C.c_void_p), int(field.nx), int(field.ny),
                          float(field.dx), float(field.dy), float(field.x0), float(field.y0),
                          float(t))


def _ptrs(arrays, dtype):
    out = (C.c_void_p * len(arrays))()
    for k, a in enumerate(arrays):
        assert a.dtype == dtype and a.flags["C_CONTIGUOUS"]
        out[k] = a.ctypes.data
    return out


def yee_advance_b(comps, dx, dy, dtb):
    """B -= dtb curl E on six float32 (ny, nx) arrays (Ex Ey Ez Bx By Bz), in place."""
    ny, nx = comps[0].shape
    lib().or_yee_advance_b(_ptrs(comps, np.float32), nx, ny, float(dx), float(dy), float(dtb))


def yee_advance_e(comps, J, dx, dy, dt):
    """E += dt (curl B - J); J: three float32 (ny, nx) arrays or None."""
    ny, nx = comps[0].shape
    lib().or_yee_advance_e(_ptrs(comps, np.float32), None if J is None else _ptrs(J, np.float32),
                           nx, ny, float(dx), float(dy), float(dt))


def deposit_current(sp: Species, q, dt, J, dx, dy, x0=0.0, y0=0.0):
    """Add the current of sp's live particles to J (three float64 (ny, nx) arrays)."""
    ny, nx = J[0].shape
    st = sp._struct()
    lib().or_deposit_current(C.byref(st), float(q), float(dt), _ptrs(J, np.float64), nx, ny,
                             float(dx), float(dy), float(x0), float(y0))


def sort_by_cell(sp: Species, nx, ny, dx, dy, x0=0.0, y0=0.0):
    st = sp._struct()
    if lib().or_sort_by_cell(C.byref(st), int(nx), int(ny), float(dx), float(dy), float(x0),
                             float(y0)) != 0:
        raise MemoryError("or_sort_by_cell")
