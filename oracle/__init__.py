"""FP64 CPU oracle of the explicit PIC cycle: a ctypes wrapper around pic_oracle.c.

TEST INFRASTRUCTURE ONLY. The tests, the smoke check and the bench's CPU baseline
are the only callers; the CUDA library never imports, links or runs anything here.

What it computes (Sec. 3 of the paper: the per-super-particle loop plus the field
update of a patch-based PIC code; the schemes are the standard published ones, the
paper identifying the field solver only as a standard second-order one, Sec. 2.1):
order-2 B-spline interpolation from the Yee grid, relativistic Boris push,
Esirkepov (2001) charge-conserving deposition, Yee (1966) FDTD, moving window.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc. FMA contraction is off so that x86 and Arm
    hosts round identically."""
    if force or not os.path.exists(_LIB_PATH) or (
        os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(_SRC),
                                           os.path.getmtime(_SRC[:-2] + ".h"))):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
               "-o", _LIB_PATH, _SRC, "-lm"]
        subprocess.check_call(cmd)
    return _LIB_PATH


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class OrcConfig(ctypes.Structure):
    _fields_ = [
        ("dims", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("d", ctypes.c_double * 3),
        ("dt", ctypes.c_double),
        ("window", ctypes.c_int),
        ("q", ctypes.c_double),
        ("m", ctypes.c_double),
        ("n0", ctypes.c_double),
        ("ramp_x0", ctypes.c_double),
        ("ramp_len", ctypes.c_double),
        ("inject_ppc", ctypes.c_int * 3),
        ("order", ctypes.c_int),
    ]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        cfgp = ctypes.POINTER(OrcConfig)
        L.orc_shape2.restype = ctypes.c_long
        L.orc_shape2.argtypes = [ctypes.c_double, _dp]
        L.orc_boris.argtypes = [ctypes.c_double] * 3 + [_dp, _dp, _dp]
        L.orc_interp.argtypes = [cfgp, ctypes.POINTER(_dp), _dp, _dp]
        L.orc_deposit.argtypes = [cfgp, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                  ctypes.POINTER(_dp)]
        L.orc_rho.argtypes = [cfgp, ctypes.c_longlong, _dp, _dp, _dp, _dp,
                              ctypes.c_double, _dp]
        L.orc_yee_e.argtypes = [cfgp, ctypes.POINTER(_dp), ctypes.POINTER(_dp),
                                ctypes.POINTER(_dp)]
        L.orc_yee_b.argtypes = [cfgp, ctypes.POINTER(_dp), ctypes.POINTER(_dp)]
        L.orc_div_e.argtypes = [cfgp, ctypes.POINTER(_dp), _dp]
        L.orc_shift_count.restype = ctypes.c_longlong
        L.orc_shift_count.argtypes = [cfgp, ctypes.c_longlong]
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [cfgp, ctypes.c_longlong]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_set_particles.argtypes = [ctypes.c_void_p, ctypes.c_longlong] + [_dp] * 7 + [_ip]
        L.orc_num_particles.restype = ctypes.c_longlong
        L.orc_num_particles.argtypes = [ctypes.c_void_p]
        L.orc_get_particles.argtypes = [ctypes.c_void_p] + [_dp] * 7 + [_ip]
        L.orc_set_fields.argtypes = [ctypes.c_void_p] + [_dp] * 6
        L.orc_get_fields.argtypes = [ctypes.c_void_p, _dp]
        L.orc_set_rho_bg.argtypes = [ctypes.c_void_p, _dp]
        L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_step_mt.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
        L.orc_steps_done.restype = ctypes.c_longlong
        L.orc_steps_done.argtypes = [ctypes.c_void_p]
        L.orc_shifts_done.restype = ctypes.c_longlong
        L.orc_shifts_done.argtypes = [ctypes.c_void_p]
        L.orc_energy.argtypes = [ctypes.c_void_p, _dp]
        L.orc_gauss.argtypes = [ctypes.c_void_p, _dp]
        L.orc_merge_group.restype = ctypes.c_int
        L.orc_merge_group.argtypes = [ctypes.c_longlong, _dp, _dp, _dp, _dp, _ip, _dp, _dp,
                                      ctypes.POINTER(ctypes.c_longlong)]
        L.orc_split.restype = ctypes.c_longlong
        L.orc_split.argtypes = [ctypes.c_void_p, _ip, ctypes.c_longlong, ctypes.c_double]
        L.orc_merge.restype = ctypes.c_longlong
        L.orc_merge.argtypes = [ctypes.c_void_p, _ip, ctypes.c_longlong, ctypes.c_double]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    if a.dtype == np.float64:
        return a.ctypes.data_as(_dp)
    if a.dtype == np.int32:
        return a.ctypes.data_as(_ip)
    raise TypeError(a.dtype)


def _arr_ptrs(arrs):
    return (_dp * len(arrs))(*[_ptr(a) for a in arrs])


def make_config(dims, n, d, dt, window=False, q=-1.0, m=1.0, n0=0.0, ramp_x0=0.0,
                ramp_len=1.0, inject_ppc=(1, 1, 1), order=2) -> OrcConfig:
    """`order`: 2 for Yee's solver, 6 for sixth-order staggered space derivatives."""
    c = OrcConfig()
    c.order = int(order)
    c.dims = dims
    n = list(n) + [1] * (3 - len(n))
    d = list(d) + [1.0] * (3 - len(d))
    for a in range(3):
        c.n[a] = int(n[a])
        c.d[a] = float(d[a])
    c.dt = float(dt)
    c.window = 1 if window else 0
    c.q, c.m = float(q), float(m)
    c.n0, c.ramp_x0, c.ramp_len = float(n0), float(ramp_x0), float(ramp_len)
    ip = list(inject_ppc) + [1] * (3 - len(inject_ppc))
    for a in range(3):
        c.inject_ppc[a] = int(ip[a])
    return c


def field_shape(c: OrcConfig):
    return (c.n[2], c.n[1], c.n[0]) if c.dims == 3 else (c.n[1], c.n[0])


# ----------------------------------------------------------------- building blocks

def shape2(xi: float):
    S = np.zeros(3)
    i = lib().orc_shape2(float(xi), _ptr(S))
    return int(i), S


def boris(q, m, dt, E, B, u):
    E = np.ascontiguousarray(E, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    u = np.array(u, dtype=np.float64)
    lib().orc_boris(q, m, dt, _ptr(E), _ptr(B), _ptr(u))
    return u


def interp(c: OrcConfig, F, pos):
    F = [np.ascontiguousarray(f, dtype=np.float64) for f in F]
    pos = np.array(list(pos) + [0.0] * (3 - len(pos)), dtype=np.float64)
    out = np.zeros(6)
    lib().orc_interp(ctypes.byref(c), _arr_ptrs(F), _ptr(pos), _ptr(out))
    return out


def deposit(c: OrcConfig, pos0, pos1, vz, qw, J):
    """Adds one particle's Esirkepov current into J (list of three arrays, in place)."""
    p0 = np.array(list(pos0) + [0.0] * (3 - len(pos0)), dtype=np.float64)
    p1 = np.array(list(pos1) + [0.0] * (3 - len(pos1)), dtype=np.float64)
    lib().orc_deposit(ctypes.byref(c), _ptr(p0), _ptr(p1), float(vz), float(qw),
                      _arr_ptrs(J))


def rho(c: OrcConfig, x, y, z, w, q):
    out = np.zeros(field_shape(c))
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    z = np.ascontiguousarray(z if z is not None else np.zeros_like(x), dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    lib().orc_rho(ctypes.byref(c), len(x), _ptr(x), _ptr(y), _ptr(z), _ptr(w), float(q),
                  _ptr(out))
    return out


def yee_e(c: OrcConfig, E, B, J):
    lib().orc_yee_e(ctypes.byref(c), _arr_ptrs(E), _arr_ptrs(B), _arr_ptrs(J))


def yee_b(c: OrcConfig, E, B):
    lib().orc_yee_b(ctypes.byref(c), _arr_ptrs(E), _arr_ptrs(B))


def div_e(c: OrcConfig, E):
    out = np.zeros(field_shape(c))
    lib().orc_div_e(ctypes.byref(c), _arr_ptrs(E), _ptr(out))
    return out


def merge_group(ux, uy, uz, w, ids):
    """Two-particle replacement of one merge group (None when fewer than 3 members):
    returns (u_a, u_b, common weight, (index of a, index of b))."""
    n = len(ux)
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (ux, uy, uz, w)]
    ida = np.ascontiguousarray(ids, dtype=np.int32)
    out = np.zeros(6)
    ow = ctypes.c_double()
    keep = (ctypes.c_longlong * 2)()
    r = lib().orc_merge_group(n, *[_ptr(a) for a in arrs], ida.ctypes.data_as(_ip), _ptr(out),
                              ctypes.byref(ow), keep)
    if r == 0:
        return None
    return out[:3].copy(), out[3:].copy(), ow.value, (int(keep[0]), int(keep[1]))


def shift_count(c: OrcConfig, step: int) -> int:
    return int(lib().orc_shift_count(ctypes.byref(c), int(step)))


# ----------------------------------------------------------------- simulation

PARTICLE_KEYS = ("x", "y", "z", "ux", "uy", "uz", "w")


class OracleSim:
    """A whole FP64 CPU simulation (test infrastructure)."""

    def __init__(self, c: OrcConfig, capacity: int):
        self.c = c
        self._h = lib().orc_create(ctypes.byref(c), int(capacity))
        if not self._h:
            raise ValueError("invalid oracle configuration")
        self.fshape = field_shape(c)
        self.ncell = int(np.prod(self.fshape))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def set_particles(self, p: dict):
        n = len(p["x"])
        arrs = [np.ascontiguousarray(p.get(k, np.zeros(n)), dtype=np.float64)
                for k in PARTICLE_KEYS]
        ids = np.ascontiguousarray(p["id"], dtype=np.int32)
        rc = lib().orc_set_particles(self._h, n, *[_ptr(a) for a in arrs], _ptr(ids))
        if rc:
            raise ValueError("particle count exceeds capacity")

    def num_particles(self) -> int:
        return int(lib().orc_num_particles(self._h))

    def get_particles(self, sort_by_id: bool = True) -> dict:
        n = self.num_particles()
        out = {k: np.zeros(n) for k in PARTICLE_KEYS}
        out["id"] = np.zeros(n, dtype=np.int32)
        lib().orc_get_particles(self._h, *[_ptr(out[k]) for k in PARTICLE_KEYS],
                                _ptr(out["id"]))
        if sort_by_id:
            order = np.argsort(out["id"], kind="stable")
            out = {k: v[order] for k, v in out.items()}
        return out

    def set_fields(self, E, B):
        arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(self.fshape)
                for a in list(E) + list(B)]
        lib().orc_set_fields(self._h, *[_ptr(a) for a in arrs])

    def get_fields(self) -> dict:
        out = np.zeros((12,) + self.fshape)
        lib().orc_get_fields(self._h, _ptr(out))
        names = ["Ex", "Ey", "Ez", "Bx", "By", "Bz", "Bnx", "Bny", "Bnz", "Jx", "Jy", "Jz"]
        return {k: out[i] for i, k in enumerate(names)}

    def set_rho_bg(self, rho_bg=None):
        if rho_bg is None:
            lib().orc_set_rho_bg(self._h, None)
        else:
            a = np.ascontiguousarray(rho_bg, dtype=np.float64)
            lib().orc_set_rho_bg(self._h, _ptr(a))

    def step(self, n: int = 1, threads: int = 1):
        """n steps; threads > 1 runs the threaded form (bit-identical results)."""
        if threads > 1:
            rc = lib().orc_step_mt(self._h, int(n), int(threads))
        else:
            rc = lib().orc_step(self._h, int(n))
        if rc:
            raise RuntimeError(f"oracle step failed ({rc})")

    @property
    def steps(self) -> int:
        return int(lib().orc_steps_done(self._h))

    @property
    def shifts(self) -> int:
        return int(lib().orc_shifts_done(self._h))

    def merge(self, patch, above: int, dp: float) -> int:
        """Merge groups (same cell and momentum bin of width dp, >= 3 members) in every
        patch holding more than `above` particles; returns the number removed."""
        pt = np.ascontiguousarray(list(patch) + [1] * (3 - len(patch)), dtype=np.int32)
        r = lib().orc_merge(self._h, pt.ctypes.data_as(_ip), int(above), float(dp))
        if r < 0:
            raise MemoryError("oracle merge")
        return int(r)

    def split(self, patch, below: int, wmin: float) -> int:
        """Split particles of cells holding fewer than `below` (and at least one)
        particles (weights >= 2 wmin, increasing id); returns the number of splits."""
        pt = np.ascontiguousarray(list(patch) + [1] * (3 - len(patch)), dtype=np.int32)
        r = lib().orc_split(self._h, pt.ctypes.data_as(_ip), int(below), float(wmin))
        if r < 0:
            raise MemoryError("oracle split (capacity)")
        return int(r)

    def energy(self):
        out = np.zeros(3)
        lib().orc_energy(self._h, _ptr(out))
        return out

    def gauss(self):
        out = np.zeros(self.fshape)
        lib().orc_gauss(self._h, _ptr(out))
        return out
