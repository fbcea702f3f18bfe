"""Thin Python binding of libvet (include/vet.h): argument marshalling only.

Every step of the closure runs in the library's CUDA kernels; this module
checks shapes and dtypes, passes raw pointers and the current CUDA stream, and
turns status codes into exceptions.  It fails loudly when the compiled library
is missing: there is no CPU fallback.

Field arguments may be CUDA torch tensors (the fast path, asynchronous on the
current stream) or host arrays (numpy or CPU torch; the library then stages
the copies itself and returns after they complete).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

VET_OK, VET_EINVAL, VET_ENOMEM, VET_ECUDA, VET_ETIMEOUT, VET_EUNSUPPORTED = range(6)
VET_FP32, VET_FP64 = 0, 1
_STATUS = {1: "VET_EINVAL", 2: "VET_ENOMEM", 3: "VET_ECUDA", 4: "VET_ETIMEOUT", 5: "VET_EUNSUPPORTED"}

#: every entry point declared in include/vet.h
EXPORTS = (
    "vet_create", "vet_destroy", "vet_num_directions", "vet_directions", "vet_trace", "vet_moments",
    "vet_closure", "vet_trace_f64", "vet_moments_f64", "vet_closure_f64", "vet_sync", "vet_work_counts",
    "vet_set_timing", "vet_last_timing", "vet_launches_per_closure", "vet_last_error", "vet_closure_noalloc",
    "vet_set_tuning", "vet_get_tuning", "vet_autotune", "vet_batch_create", "vet_batch_destroy", "vet_batch_context",
    "vet_batch_closure", "vet_batch_sync", "vet_batch_autotune", "vet_batch_last_error",
)


class VetError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("block", ctypes.c_int),
                ("h", ctypes.c_double)]


class _Config(ctypes.Structure):
    _fields_ = [("nside", ctypes.c_int), ("rot_q", ctypes.c_double * 4), ("precision", ctypes.c_int),
                ("device", ctypes.c_int), ("spin_limit", ctypes.c_longlong)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libvet (building it first if asked and needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libvet is not built ({path} missing); run paper_2202_08778_gb300.build.build()")
        lib = ctypes.CDLL(path)
        vp, i = ctypes.c_void_p, ctypes.c_int
        lib.vet_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_Grid), ctypes.POINTER(_Config)]
        lib.vet_destroy.argtypes = [vp]
        lib.vet_num_directions.argtypes = [vp]
        lib.vet_num_directions.restype = i
        lib.vet_directions.argtypes = [vp, vp]
        for name in ("vet_trace", "vet_trace_f64"):
            getattr(lib, name).argtypes = [vp, vp, vp, vp, vp, vp]
        for name in ("vet_moments", "vet_moments_f64"):
            getattr(lib, name).argtypes = [vp, vp, vp, vp]
        for name in ("vet_closure", "vet_closure_f64"):
            getattr(lib, name).argtypes = [vp, vp, vp, vp, vp, vp, vp]
        lib.vet_sync.argtypes = [vp]
        lib.vet_work_counts.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
        lib.vet_set_timing.argtypes = [vp, i]
        lib.vet_last_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
        lib.vet_launches_per_closure.argtypes = [vp]
        lib.vet_launches_per_closure.restype = i
        lib.vet_closure_noalloc.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Config), vp, vp, vp, vp, vp, vp]
        ip = ctypes.POINTER(ctypes.c_int)
        lib.vet_set_tuning.argtypes = [vp, i, i]
        lib.vet_get_tuning.argtypes = [vp, ip, ip]
        lib.vet_autotune.argtypes = [vp, vp, vp, vp, ip, ip, vp]
        lib.vet_batch_create.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(_Grid), ctypes.POINTER(_Config)]
        lib.vet_batch_destroy.argtypes = [vp]
        lib.vet_batch_context.argtypes = [vp, i]
        lib.vet_batch_context.restype = vp
        lib.vet_batch_closure.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        lib.vet_batch_sync.argtypes = [vp]
        lib.vet_batch_autotune.argtypes = [vp, vp, vp, vp, vp]
        lib.vet_batch_last_error.argtypes = [vp]
        lib.vet_batch_last_error.restype = ctypes.c_char_p
        lib.vet_last_error.argtypes = [vp]
        lib.vet_last_error.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name not in ("vet_num_directions", "vet_last_error", "vet_launches_per_closure", "vet_batch_context",
                            "vet_batch_last_error"):
                getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _ptr(a, dtype, n, name):
    """Raw pointer of a torch tensor or numpy array after shape/dtype checks."""
    if a is None:
        return None
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(a, torch.Tensor):
        want = torch.float32 if dtype == np.float32 else torch.float64
        if a.dtype != want:
            raise TypeError(f"{name}: expected {want}, got {a.dtype}")
        if not a.is_contiguous():
            raise ValueError(f"{name}: tensor must be contiguous")
        if a.numel() != n:
            raise ValueError(f"{name}: expected {n} elements, got {a.numel()}")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if a.dtype != dtype:
            raise TypeError(f"{name}: expected {np.dtype(dtype)}, got {a.dtype}")
        if not a.flags.c_contiguous:
            raise ValueError(f"{name}: array must be C-contiguous")
        if a.size != n:
            raise ValueError(f"{name}: expected {n} elements, got {a.size}")
        return a.ctypes.data
    raise TypeError(f"{name}: expected a torch tensor or a numpy array, got {type(a).__name__}")


def _stream(stream):
    if stream is not None:
        return int(stream)
    try:
        import torch

        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:  # pragma: no cover
        pass
    return None


class Context:
    """A libvet context: grid, direction set, templates and workspace."""

    def __init__(self, shape, block: int, h: float, nside: int, rot_q=(1.0, 0.0, 0.0, 0.0),
                 precision: int = VET_FP32, device: int = 0, spin_limit: int = 0):
        self._lib = load()
        nz, ny, nx = shape
        self.shape = (int(nz), int(ny), int(nx))
        self.ncell = int(nz) * int(ny) * int(nx)
        self.precision = precision
        self.dtype = np.float64 if precision == VET_FP64 else np.float32
        g = _Grid(int(nx), int(ny), int(nz), int(block), float(h))
        q = (ctypes.c_double * 4)(*[float(v) for v in rot_q])
        cfg = _Config(int(nside), q, int(precision), int(device), int(spin_limit))
        h_ = ctypes.c_void_p()
        st = self._lib.vet_create(ctypes.byref(h_), ctypes.byref(g), ctypes.byref(cfg))
        if st != VET_OK:
            raise VetError(st, self._lib.vet_last_error(None).decode())
        self._h = h_
        self.N = self._lib.vet_num_directions(self._h)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.vet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != VET_OK:
            raise VetError(st, self._lib.vet_last_error(self._h).decode())

    def directions(self) -> np.ndarray:
        out = np.zeros((self.N, 4), dtype=np.float64)
        self._check(self._lib.vet_directions(self._h, out.ctypes.data))
        return out

    def work_counts(self):
        a, b = ctypes.c_longlong(), ctypes.c_longlong()
        self._check(self._lib.vet_work_counts(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def _fn(self, base):
        return getattr(self._lib, base + ("_f64" if self.precision == VET_FP64 else ""))

    def trace(self, kappa, S, Ib, I_out, stream=None):
        nc, dt = self.ncell, self.dtype
        self._check(self._fn("vet_trace")(self._h, _ptr(kappa, dt, nc, "kappa"), _ptr(S, dt, nc, "S"),
                                          _ptr(Ib, dt, 6 * self.N, "Ib"), _ptr(I_out, dt, self.N * nc, "I_out"),
                                          _stream(stream)))
        return I_out

    def moments(self, I, M_out, stream=None):
        nc, dt = self.ncell, self.dtype
        self._check(self._fn("vet_moments")(self._h, _ptr(I, dt, self.N * nc, "I"), _ptr(M_out, dt, 10 * nc, "M_out"),
                                            _stream(stream)))
        return M_out

    def closure(self, kappa, S, Ib, f_out, M_out=None, stream=None):
        nc, dt = self.ncell, self.dtype
        self._check(self._fn("vet_closure")(self._h, _ptr(kappa, dt, nc, "kappa"), _ptr(S, dt, nc, "S"),
                                            _ptr(Ib, dt, 6 * self.N, "Ib"), _ptr(f_out, dt, 6 * nc, "f_out"),
                                            _ptr(M_out, dt, 10 * nc, "M_out"), _stream(stream)))
        return f_out

    def set_timing(self, enable: bool = True):
        self._check(self._lib.vet_set_timing(self._h, int(bool(enable))))

    def last_timing(self):
        """(face pass, cell pass, closing step, whole call) in ms of the last call."""
        ms = (ctypes.c_float * 4)()
        self._check(self._lib.vet_last_timing(self._h, ms))
        return tuple(float(v) for v in ms)

    def launches_per_closure(self) -> int:
        return int(self._lib.vet_launches_per_closure(self._h))

    def sync(self):
        self._check(self._lib.vet_sync(self._h))

    def set_tuning(self, face_group: int = 0, dir_tile: int = 0):
        self._check(self._lib.vet_set_tuning(self._h, int(face_group), int(dir_tile)))

    def tuning(self):
        fg, dt = ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.vet_get_tuning(self._h, ctypes.byref(fg), ctypes.byref(dt)))
        return fg.value, dt.value

    def autotune(self, kappa, S, Ib=None, stream=None):
        """Time the candidate tunings on these device inputs; keep the fastest."""
        nc = self.ncell
        fg, dt = ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.vet_autotune(self._h, _ptr(kappa, np.float32, nc, "kappa"), _ptr(S, np.float32, nc, "S"),
                                           _ptr(Ib, np.float32, 6 * self.N, "Ib"), ctypes.byref(fg),
                                           ctypes.byref(dt), _stream(stream)))
        return fg.value, dt.value


def closure_noalloc(shape, block: int, h: float, nside: int, kappa, S, Ib, f_out, M_out=None,
                    rot_q=(1.0, 0.0, 0.0, 0.0), device: int = 0, spin_limit: int = 0, stream=None):
    """vet_closure_noalloc: the FP32 closure without a context and without any
    allocation (workspace is a static device array inside libvet; see
    include/vet.h for its limits).  Field arguments must be CUDA tensors."""
    lib = load()
    nz, ny, nx = shape
    n = int(nz) * int(ny) * int(nx)
    N = 12 * int(nside) ** 2
    g = _Grid(int(nx), int(ny), int(nz), int(block), float(h))
    q = (ctypes.c_double * 4)(*[float(v) for v in rot_q])
    cfg = _Config(int(nside), q, VET_FP32, int(device), int(spin_limit))
    st = lib.vet_closure_noalloc(ctypes.byref(g), ctypes.byref(cfg), _ptr(kappa, np.float32, n, "kappa"),
                                 _ptr(S, np.float32, n, "S"), _ptr(Ib, np.float32, 6 * N, "Ib"),
                                 _ptr(f_out, np.float32, 6 * n, "f_out"), _ptr(M_out, np.float32, 10 * n, "M_out"),
                                 _stream(stream))
    if st != VET_OK:
        raise VetError(st, lib.vet_last_error(None).decode())
    return f_out


class _Member(Context):
    """A grid of a Batch: a view of a context the batch owns."""

    def __init__(self, lib, handle, shape):
        self._lib = lib
        self._h = ctypes.c_void_p(handle)
        self.shape = tuple(int(v) for v in shape)
        self.ncell = int(np.prod(self.shape))
        self.precision = VET_FP32
        self.dtype = np.float32
        self.N = lib.vet_num_directions(self._h)

    def close(self):  # owned by the batch
        self._h = None


class Batch:
    """vet_batch: independent grids whose closures run as one CUDA graph
    (one branch per grid).  problems: list of (shape, block, h, nside, rot_q)."""

    def __init__(self, problems, device: int = 0, spin_limit: int = 0):
        self._lib = load()
        n = len(problems)
        grids = (_Grid * n)()
        cfgs = (_Config * n)()
        for i, (shape, block, h, nside, q) in enumerate(problems):
            nz, ny, nx = shape
            grids[i] = _Grid(int(nx), int(ny), int(nz), int(block), float(h))
            cfgs[i] = _Config(int(nside), (ctypes.c_double * 4)(*[float(v) for v in q]), VET_FP32, int(device),
                              int(spin_limit))
        h_ = ctypes.c_void_p()
        st = self._lib.vet_batch_create(ctypes.byref(h_), n, grids, cfgs)
        if st != VET_OK:
            raise VetError(st, self._lib.vet_last_error(None).decode())
        self._h = h_
        self.n = n
        self.members = [_Member(self._lib, self._lib.vet_batch_context(self._h, i), problems[i][0]) for i in range(n)]

    def close(self):
        if getattr(self, "_h", None):
            for m in self.members:
                m.close()
            self._lib.vet_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != VET_OK:
            raise VetError(st, self._lib.vet_batch_last_error(self._h).decode())

    def _arr(self, xs, sizes, name, allow_none=False):
        if xs is None:
            return None
        arr = (ctypes.c_void_p * self.n)()
        for i, (x, n) in enumerate(zip(xs, sizes)):
            if x is None and allow_none:
                arr[i] = None
            else:
                arr[i] = _ptr(x, np.float32, n, f"{name}[{i}]")
        return arr

    def closure(self, kappa, S, Ib, f_out, M_out=None, stream=None):
        nc = [m.ncell for m in self.members]
        self._check(self._lib.vet_batch_closure(
            self._h, self._arr(kappa, nc, "kappa"), self._arr(S, nc, "S"),
            self._arr(Ib, [6 * m.N for m in self.members], "Ib", True), self._arr(f_out, [6 * c for c in nc], "f_out"),
            self._arr(M_out, [10 * c for c in nc], "M_out", True), _stream(stream)))

    def autotune(self, kappa, S, Ib=None, stream=None):
        nc = [m.ncell for m in self.members]
        self._check(self._lib.vet_batch_autotune(self._h, self._arr(kappa, nc, "kappa"), self._arr(S, nc, "S"),
                                                 self._arr(Ib, [6 * m.N for m in self.members], "Ib", True),
                                                 _stream(stream)))

    def sync(self):
        self._check(self._lib.vet_batch_sync(self._h))
