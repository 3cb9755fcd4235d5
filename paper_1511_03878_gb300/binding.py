"""Thin ctypes binding of libpic.so (include/pic.h): same names, argument
marshalling only. Every step of the PIC cycle runs in the CUDA library; there is
no CPU fallback - if the library or a GPU is missing, calls raise.

PyTorch provides the device arena (a uint8 tensor) and the CUDA stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpic.so")

PIC_OK, PIC_ERR_INVALID, PIC_ERR_NOMEM, PIC_ERR_CAPACITY = 0, -1, -2, -3
PIC_ERR_CUDA, PIC_ERR_NUMERIC, PIC_ERR_TIMEOUT = -4, -5, -6
PIC_FP64, PIC_FP32, PIC_DF64 = 0, 1, 2
PIC_MAP_QUEUE, PIC_MAP_STATIC = 0, 1
(PIC_DIAG_ENERGY, PIC_DIAG_GAUSS, PIC_DIAG_FIELDS, PIC_DIAG_PARTICLES,
 PIC_DIAG_NUM_PARTICLES, PIC_DIAG_PATCH_COUNTS, PIC_DIAG_STEP, PIC_DIAG_EX_AXIS,
 PIC_DIAG_QUEUE, PIC_DIAG_SLOTS) = range(10)

STATUS_NAMES = {0: "PIC_OK", -1: "PIC_ERR_INVALID", -2: "PIC_ERR_NOMEM",
                -3: "PIC_ERR_CAPACITY", -4: "PIC_ERR_CUDA", -5: "PIC_ERR_NUMERIC",
                -6: "PIC_ERR_TIMEOUT"}

# every symbol include/pic.h declares
EXPORTS = ("pic_config_bytes", "pic_required_bytes", "pic_create", "pic_load_particles", "pic_load_fields",
           "pic_step", "pic_sync", "pic_diag", "pic_step_record_async", "pic_record_wait",
           "pic_profile", "pic_destroy", "pic_last_error",
           "pic_batch_required_bytes", "pic_batch_create", "pic_batch_step",
           "pic_batch_destroy", "pic_gauss_residual_2d_static", "pic_selftest_bounded_wait",
           "pic_hilbert_order", "pic_partition")
PIC_STATIC_MAX_CELLS = 1 << 20


class PicError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class PicConfig(ctypes.Structure):
    _fields_ = [
        ("dims", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("d", ctypes.c_double * 3),
        ("dt", ctypes.c_double),
        ("patch", ctypes.c_int * 3),
        ("precision", ctypes.c_int),
        ("window", ctypes.c_int),
        ("n0", ctypes.c_double),
        ("ramp_x0", ctypes.c_double),
        ("ramp_len", ctypes.c_double),
        ("inject_ppc", ctypes.c_int * 3),
        ("q", ctypes.c_double),
        ("m", ctypes.c_double),
        ("capacity", ctypes.c_longlong),
        ("chunk", ctypes.c_int),
        ("mapping", ctypes.c_int),
        ("merge_above", ctypes.c_int),
        ("merge_dp", ctypes.c_double),
        ("maxwell_order", ctypes.c_int),
        ("split_below", ctypes.c_int),
        ("split_wmin", ctypes.c_double),
    ]


_lib = None


def lib():
    """Loads libpic.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
        L = ctypes.CDLL(LIB_PATH)
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
        cfgp = ctypes.POINTER(PicConfig)
        L.pic_config_bytes.restype = ctypes.c_size_t
        L.pic_config_bytes.argtypes = []
        if L.pic_config_bytes() != ctypes.sizeof(PicConfig):
            raise RuntimeError(f"{LIB_PATH} was built with a different pic_config layout "
                               f"({L.pic_config_bytes()} bytes, binding {ctypes.sizeof(PicConfig)})")
        L.pic_required_bytes.restype = ctypes.c_size_t
        L.pic_required_bytes.argtypes = [cfgp]
        L.pic_create.restype = ctypes.c_int
        L.pic_create.argtypes = [cfgp, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]
        L.pic_load_particles.restype = ctypes.c_int
        L.pic_load_particles.argtypes = [vp, ctypes.c_longlong] + [dp] * 7 + [ip]
        L.pic_load_fields.restype = ctypes.c_int
        L.pic_load_fields.argtypes = [vp, ctypes.POINTER(dp), ctypes.POINTER(dp), dp]
        L.pic_step.restype = ctypes.c_int
        L.pic_step.argtypes = [vp, ctypes.c_int]
        L.pic_sync.restype = ctypes.c_int
        L.pic_sync.argtypes = [vp]
        L.pic_diag.restype = ctypes.c_int
        L.pic_diag.argtypes = [vp, ctypes.c_int, vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
        L.pic_step_record_async.restype = ctypes.c_int
        L.pic_step_record_async.argtypes = [vp, ctypes.c_int]
        L.pic_record_wait.restype = ctypes.c_int
        L.pic_record_wait.argtypes = [vp, ctypes.c_int, vp, ctypes.c_size_t,
                                      ctypes.POINTER(ctypes.c_size_t)]
        L.pic_profile.restype = ctypes.c_int
        L.pic_profile.argtypes = [vp, ctypes.c_int, dp, ctypes.c_int]
        L.pic_destroy.restype = ctypes.c_int
        L.pic_destroy.argtypes = [vp]
        L.pic_last_error.restype = ctypes.c_char_p
        L.pic_last_error.argtypes = [vp]
        L.pic_batch_required_bytes.restype = ctypes.c_size_t
        L.pic_batch_required_bytes.argtypes = [ctypes.POINTER(vp), ctypes.c_int]
        L.pic_batch_create.restype = ctypes.c_int
        L.pic_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp, ctypes.c_size_t, vp,
                                       ctypes.POINTER(vp)]
        L.pic_batch_step.restype = ctypes.c_int
        L.pic_batch_step.argtypes = [vp, ctypes.c_int]
        L.pic_batch_destroy.restype = ctypes.c_int
        L.pic_batch_destroy.argtypes = [vp]
        L.pic_selftest_bounded_wait.restype = ctypes.c_int
        L.pic_selftest_bounded_wait.argtypes = [vp]
        L.pic_hilbert_order.restype = ctypes.c_int
        L.pic_hilbert_order.argtypes = [ctypes.c_int, ip, ip]
        L.pic_partition.restype = ctypes.c_int
        L.pic_partition.argtypes = [ctypes.c_int, dp, ctypes.c_int, ip, dp]
        L.pic_gauss_residual_2d_static.restype = ctypes.c_int
        L.pic_gauss_residual_2d_static.argtypes = (
            [ctypes.c_longlong, vp, vp, vp, ctypes.c_double, vp, vp, vp, vp, ctypes.c_int,
             ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, vp])
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _check(rc, handle=None):
    if rc != PIC_OK:
        msg = lib().pic_last_error(handle).decode() if handle else ""
        raise PicError(rc, msg)


# ------------------------------------------------------------------ same-name wrappers

def make_config(params: dict, precision: int = PIC_FP64, capacity: int = 0, chunk: int = 0,
                mapping: int = PIC_MAP_QUEUE, merge_above: int = 0,
                merge_dp: float = 0.0, split_below: int = 0,
                split_wmin: float = 0.0) -> PicConfig:
    c = PicConfig()
    c.dims = int(params["dims"])
    for a in range(3):
        c.n[a] = int(params["n"][a]) if a < len(params["n"]) else 1
        c.d[a] = float(params["d"][a]) if a < len(params["d"]) else 1.0
        pt = params.get("patch", (32, 32, 32))
        c.patch[a] = int(pt[a]) if a < len(pt) else 1
        ip = params.get("inject_ppc", (1, 1, 1))
        c.inject_ppc[a] = int(ip[a]) if a < len(ip) else 1
    if c.dims == 2:
        c.n[2] = 1
    c.dt = float(params["dt"])
    c.precision = int(precision)
    c.window = 1 if params.get("window") else 0
    c.n0 = float(params.get("n0", 0.0))
    c.ramp_x0 = float(params.get("ramp_x0", 0.0))
    c.ramp_len = float(params.get("ramp_len", 1.0))
    c.q = float(params.get("q", -1.0))
    c.m = float(params.get("m", 1.0))
    c.capacity = int(capacity)
    c.chunk = int(chunk)
    c.mapping = int(mapping)
    c.merge_above = int(merge_above)
    c.merge_dp = float(merge_dp)
    c.maxwell_order = int(params.get("maxwell_order", 2))
    c.split_below = int(split_below)
    c.split_wmin = float(split_wmin)
    return c


def pic_config_bytes() -> int:
    return int(lib().pic_config_bytes())


def pic_required_bytes(cfg: PicConfig) -> int:
    return int(lib().pic_required_bytes(ctypes.byref(cfg)))


# cells of the grid of every live handle made by pic_create (the library reads that
# many values from each host field array)
_ncell = {}


def pic_create(cfg: PicConfig, arena_ptr: int, arena_bytes: int, stream_ptr: int):
    h = ctypes.c_void_p()
    _check(lib().pic_create(ctypes.byref(cfg), ctypes.c_void_p(arena_ptr), arena_bytes,
                            ctypes.c_void_p(stream_ptr), ctypes.byref(h)))
    _ncell[h.value] = int(cfg.n[0]) * int(cfg.n[1]) * (int(cfg.n[2]) if cfg.dims == 3 else 1)
    return h


def _check_particles(p: dict) -> int:
    """n from x; every other array given (ids required) must hold n entries, since the
    library reads n values from each pointer."""
    n = int(np.size(p["x"]))
    if "id" not in p:
        raise ValueError("particle ids are required")
    for k in ("y", "z", "ux", "uy", "uz", "w", "id"):
        if k in p and np.size(p[k]) != n:
            raise ValueError(f"particle array {k!r} has {np.size(p[k])} entries, x has {n}")
    return n


def _check_fields(h, E, B, rho_bg):
    """Three components each for E and B, all (and rho_bg) with the grid's cell count."""
    ncell = _ncell.get(h.value if isinstance(h, ctypes.c_void_p) else h)
    for name, arrs in (("E", E), ("B", B)):
        if len(arrs) != 3:
            raise ValueError(f"{name} needs three components, got {len(arrs)}")
    sizes = [np.size(a) for a in list(E) + list(B)]
    if rho_bg is not None:
        sizes.append(np.size(rho_bg))
    want = ncell if ncell is not None else sizes[0]
    for k, sz in enumerate(sizes):
        if sz != want:
            what = ("E", "B")[k // 3] + f"[{k % 3}]" if k < 6 else "rho_bg"
            raise ValueError(f"{what} has {sz} values, the grid {want}")


def pic_load_particles(h, p: dict):
    n = _check_particles(p)
    # an absent z is passed as NULL (2D); other absent arrays as zeros, built only then
    arrs = [np.ascontiguousarray(p[k], dtype=np.float64) if k in p
            else (None if k == "z" else np.zeros(n))
            for k in ("x", "y", "z", "ux", "uy", "uz", "w")]
    ids = np.ascontiguousarray(p["id"], dtype=np.int32)
    _check(lib().pic_load_particles(h, n, *[_dp(a) for a in arrs], _ip(ids)), h)


def pic_load_fields(h, E, B, rho_bg=None):
    _check_fields(h, E, B, rho_bg)
    E = [np.ascontiguousarray(a, dtype=np.float64) for a in E]
    B = [np.ascontiguousarray(a, dtype=np.float64) for a in B]
    Ep = (ctypes.POINTER(ctypes.c_double) * 3)(*[_dp(a) for a in E])
    Bp = (ctypes.POINTER(ctypes.c_double) * 3)(*[_dp(a) for a in B])
    rb = np.ascontiguousarray(rho_bg, dtype=np.float64) if rho_bg is not None else None
    _check(lib().pic_load_fields(h, Ep, Bp, _dp(rb)), h)


def pic_step(h, nsteps: int):
    _check(lib().pic_step(h, int(nsteps)), h)


def pic_sync(h):
    _check(lib().pic_sync(h), h)


def pic_diag(h, kind: int, nbytes: int) -> bytes:
    buf = ctypes.create_string_buffer(nbytes)
    written = ctypes.c_size_t(0)
    _check(lib().pic_diag(h, kind, buf, nbytes, ctypes.byref(written)), h)
    return buf.raw[: written.value]


def pic_step_record_async(h, slot: int):
    _check(lib().pic_step_record_async(h, int(slot)), h)


def pic_record_wait(h, slot: int, nbytes: int = 24) -> bytes:
    buf = ctypes.create_string_buffer(nbytes)
    written = ctypes.c_size_t(0)
    _check(lib().pic_record_wait(h, int(slot), buf, nbytes, ctypes.byref(written)), h)
    return buf.raw[: written.value]


PROFILE_KERNELS = ("queue_build", "push", "inject", "exchange", "repack", "yee", "end_step",
                   "step")


def pic_profile(h, nsteps: int) -> dict:
    ms = np.zeros(len(PROFILE_KERNELS))
    _check(lib().pic_profile(h, int(nsteps), _dp(ms), len(PROFILE_KERNELS)), h)
    return dict(zip(PROFILE_KERNELS, ms.tolist()))


def pic_destroy(h):
    _ncell.pop(h.value if isinstance(h, ctypes.c_void_p) else h, None)
    _check(lib().pic_destroy(h))


def pic_last_error(h) -> str:
    return lib().pic_last_error(h).decode()


def pic_batch_required_bytes(handles) -> int:
    arr = (ctypes.c_void_p * len(handles))(*[h.value for h in handles])
    return int(lib().pic_batch_required_bytes(arr, len(handles)))


def pic_batch_create(handles, arena_ptr: int, arena_bytes: int, stream_ptr: int):
    arr = (ctypes.c_void_p * len(handles))(*[h.value for h in handles])
    b = ctypes.c_void_p()
    _check(lib().pic_batch_create(arr, len(handles), ctypes.c_void_p(arena_ptr), arena_bytes,
                                  ctypes.c_void_p(stream_ptr), ctypes.byref(b)))
    return b


def pic_batch_step(b, nsteps: int):
    _check(lib().pic_batch_step(b, int(nsteps)))


def pic_batch_destroy(b):
    _check(lib().pic_batch_destroy(b))


def pic_selftest_bounded_wait(stream_ptr: int) -> int:
    """Runs the bounded-wait self-test on a stream; returns the pic_status code
    (PIC_ERR_TIMEOUT is the expected outcome, see include/pic.h)."""
    return int(lib().pic_selftest_bounded_wait(ctypes.c_void_p(stream_ptr)))


def pic_gauss_residual_2d_static(n, x_ptr, y_ptr, w_ptr, q, ex_ptr, ey_ptr, rho_bg_ptr, out_ptr,
                                 nx, ny, dx, dy, window, stream_ptr) -> int:
    """Allocation-free Gauss residual on caller-owned device pointers (ints); returns
    the pic_status code (the call allocates nothing, see include/pic.h)."""
    vp = ctypes.c_void_p
    return int(lib().pic_gauss_residual_2d_static(
        int(n), vp(x_ptr), vp(y_ptr), vp(w_ptr), float(q), vp(ex_ptr), vp(ey_ptr),
        vp(rho_bg_ptr) if rho_bg_ptr else None, vp(out_ptr), int(nx), int(ny), float(dx),
        float(dy), int(window), vp(stream_ptr) if stream_ptr else None))


def pic_hilbert_order(dims: int, np_patches) -> np.ndarray:
    """Patch indices (x fastest) in Hilbert-curve order (host only)."""
    n3 = np.ascontiguousarray(list(np_patches) + [1] * (3 - len(np_patches)), dtype=np.int32)
    out = np.zeros(int(np.prod(n3[:dims])), dtype=np.int32)
    _check(lib().pic_hilbert_order(int(dims), _ip(n3), _ip(out)))
    return out


def pic_partition(load, nranks: int):
    """Contiguous segments of `load` (curve order) for `nranks` ranks with the smallest
    largest segment load (host only): returns (first[nranks + 1], max_load)."""
    load = np.ascontiguousarray(load, dtype=np.float64)
    first = np.zeros(nranks + 1, dtype=np.int32)
    mx = ctypes.c_double(0.0)
    _check(lib().pic_partition(len(load), _dp(load), int(nranks), _ip(first), ctypes.byref(mx)))
    return first, mx.value


def check_workload(workload: dict, ncell: int, rho_bg=None):
    """Raises ValueError unless the arrays have the sizes the C ABI reads: every particle
    array given as long as x (ids required), and E, B (three arrays each) and rho_bg with
    ncell values. The library reads exactly those counts from the host pointers."""
    p = workload["particles"]
    n = len(p["x"])
    for k in ("x", "y", "z", "ux", "uy", "uz", "w", "id"):
        if k not in p and k != "id":  # the loader passes zeros for an absent array
            continue
        if np.size(p[k]) != n:
            raise ValueError(f"particle array {k!r} has {np.size(p[k])} entries, x has {n}")
    for name in ("E", "B"):
        arrs = workload[name]
        if len(arrs) != 3:
            raise ValueError(f"{name} needs three components, got {len(arrs)}")
        for a, arr in enumerate(arrs):
            if np.size(arr) != ncell:
                raise ValueError(f"{name}[{a}] has {np.size(arr)} values, the grid {ncell}")
    if rho_bg is not None and np.size(rho_bg) != ncell:
        raise ValueError(f"rho_bg has {np.size(rho_bg)} values, the grid {ncell}")


# ------------------------------------------------------------------ convenience object

class Sim:
    """One simulation resident on the GPU: arena from torch, work on a torch stream."""

    def __init__(self, params: dict, precision: int = PIC_FP64, capacity: int = 0,
                 chunk: int = 0, mapping: int = PIC_MAP_QUEUE, stream=None, device="cuda",
                 merge_above: int = 0, merge_dp: float = 0.0, split_below: int = 0,
                 split_wmin: float = 0.0):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA GPU is required (the library has no CPU path)")
        self.params = params
        self.cfg = make_config(params, precision, capacity, chunk, mapping, merge_above, merge_dp,
                               split_below, split_wmin)
        self.nbytes = pic_required_bytes(self.cfg)
        if self.nbytes == 0:
            raise PicError(PIC_ERR_INVALID, "invalid configuration")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.arena = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=device)
        ptr = self.arena.data_ptr()
        ptr = (ptr + 255) // 256 * 256
        self.h = pic_create(self.cfg, ptr, self.nbytes, self.stream.cuda_stream)
        n = self.cfg.n
        self.fshape = (n[2], n[1], n[0]) if self.cfg.dims == 3 else (n[1], n[0])
        self.ncell = int(np.prod(self.fshape))
        self.npatch = int(np.prod([n[a] // self.cfg.patch[a] for a in range(self.cfg.dims)]))

    def close(self):
        """Destroys the sim (after its stream drains) and releases its arena."""
        if getattr(self, "h", None) is not None and self.h.value:
            pic_destroy(self.h)
            self.h = None
        self.arena = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load(self, workload: dict, rho_bg=None):
        check_workload(workload, self.ncell, rho_bg)
        pic_load_particles(self.h, workload["particles"])
        pic_load_fields(self.h, workload["E"], workload["B"], rho_bg)

    def step(self, n: int = 1):
        pic_step(self.h, n)

    def sync(self):
        pic_sync(self.h)

    def profile(self, nsteps: int) -> dict:
        return pic_profile(self.h, nsteps)

    def energy(self):
        return np.frombuffer(pic_diag(self.h, PIC_DIAG_ENERGY, 24), dtype=np.float64).copy()

    def gauss(self):
        b = pic_diag(self.h, PIC_DIAG_GAUSS, 8 * self.ncell)
        return np.frombuffer(b, dtype=np.float64).reshape(self.fshape).copy()

    def fields(self) -> dict:
        b = pic_diag(self.h, PIC_DIAG_FIELDS, 12 * 8 * self.ncell)
        a = np.frombuffer(b, dtype=np.float64).reshape((12,) + self.fshape)
        names = ["Ex", "Ey", "Ez", "Bx", "By", "Bz", "Bnx", "Bny", "Bnz", "Jx", "Jy", "Jz"]
        return {k: a[i].copy() for i, k in enumerate(names)}

    def num_particles(self) -> int:
        return int(np.frombuffer(pic_diag(self.h, PIC_DIAG_NUM_PARTICLES, 8), dtype=np.int64)[0])

    def particles(self) -> dict:
        n = self.num_particles()
        b = pic_diag(self.h, PIC_DIAG_PARTICLES, n * 60)
        d = np.frombuffer(b[: 56 * n], dtype=np.float64).reshape(7, n)
        out = {k: d[i].copy() for i, k in enumerate(("x", "y", "z", "ux", "uy", "uz", "w"))}
        out["id"] = np.frombuffer(b[56 * n:], dtype=np.int32).copy()
        return out

    def patch_counts(self):
        return np.frombuffer(pic_diag(self.h, PIC_DIAG_PATCH_COUNTS, 4 * self.npatch),
                             dtype=np.int32).copy()

    def step_info(self):
        s, k, _ = np.frombuffer(pic_diag(self.h, PIC_DIAG_STEP, 24), dtype=np.int64)
        return int(s), int(k)

    def step_record_async(self, slot: int):
        """Enqueue a copy of the step record into slot 0 or 1 without waiting."""
        pic_step_record_async(self.h, slot)

    def record_wait(self, slot: int):
        """Wait for the record enqueued in `slot`: (steps taken, window shifts)."""
        s, k, _ = np.frombuffer(pic_record_wait(self.h, slot), dtype=np.int64)
        return int(s), int(k)

    def merged(self) -> int:
        """Particles removed by merging so far."""
        return int(np.frombuffer(pic_diag(self.h, PIC_DIAG_STEP, 32), dtype=np.int64)[3])

    def split_count(self) -> int:
        """Particles added by splitting so far."""
        return int(np.frombuffer(pic_diag(self.h, PIC_DIAG_STEP, 40), dtype=np.int64)[4])

    def repacks(self) -> int:
        return int(np.frombuffer(pic_diag(self.h, PIC_DIAG_STEP, 24), dtype=np.int64)[2])

    def queue(self):
        """The last step's work items as an (m, 4) int32 array {sim, patch, first, count}."""
        cap = 4 + 16 * (2 * self.npatch + int(self.cfg.capacity) // max(1, self.chunk_used()) + 64)
        b = pic_diag(self.h, PIC_DIAG_QUEUE, cap)
        m = int(np.frombuffer(b[:4], dtype=np.int32)[0])
        return np.frombuffer(b[4:4 + 16 * m], dtype=np.int32).reshape(m, 4).copy()

    def slots(self):
        """Each particle's slot within its patch, in id order (as particles())."""
        n = self.num_particles()
        return np.frombuffer(pic_diag(self.h, PIC_DIAG_SLOTS, 4 * n), dtype=np.int32).copy()

    def chunk_used(self) -> int:
        return int(self.cfg.chunk) if self.cfg.chunk > 0 else 2048

    def ex_axis(self):
        return np.frombuffer(pic_diag(self.h, PIC_DIAG_EX_AXIS, 8 * self.cfg.n[0]),
                             dtype=np.float64).copy()
