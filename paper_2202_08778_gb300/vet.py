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
    "vet_model_create", "vet_model_destroy", "vet_model_num_params", "vet_model_set_params", "vet_model_get_params",
    "vet_model_get_grads", "vet_model_features", "vet_model_forward", "vet_model_backward", "vet_model_step",
    "vet_closure_learned", "vet_model_last_timing", "vet_model_last_indicator", "vet_model_last_error",
    "vet_local_closure", "vet_point_source", "vet_field_change", "vet_reuse_decision", "vet_model_save",
    "vet_model_load", "vet_hlle_wavespeed",
)

#: functions whose return value is not a vet_status
_NOT_STATUS = ("vet_num_directions", "vet_last_error", "vet_launches_per_closure", "vet_batch_context",
               "vet_batch_last_error", "vet_model_num_params", "vet_model_last_error")


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
        ip = ctypes.POINTER(ctypes.c_int)
        lib.vet_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_Grid), ctypes.POINTER(_Config)]
        lib.vet_destroy.argtypes = [vp]
        lib.vet_num_directions.argtypes = [vp]
        lib.vet_num_directions.restype = i
        lib.vet_directions.argtypes = [vp, vp]
        for name in ("vet_trace", "vet_trace_f64"):
            getattr(lib, name).argtypes = [vp, vp, vp, vp, vp, vp]
        lib.vet_moments.argtypes = [vp, vp, vp, vp, vp]
        lib.vet_moments_f64.argtypes = [vp, vp, vp, vp]
        for name in ("vet_closure", "vet_closure_f64"):
            getattr(lib, name).argtypes = [vp, vp, vp, vp, vp, vp, vp]
        lib.vet_sync.argtypes = [vp]
        lib.vet_work_counts.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
        lib.vet_set_timing.argtypes = [vp, i]
        lib.vet_last_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
        lib.vet_launches_per_closure.argtypes = [vp]
        lib.vet_launches_per_closure.restype = i
        lib.vet_closure_noalloc.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Config), vp, vp, vp, vp, vp, vp]
        lib.vet_set_tuning.argtypes = [vp, i, i]
        lib.vet_reuse_decision.argtypes = [ctypes.POINTER(ctypes.c_float), i, i, ctypes.c_double, ctypes.c_double, i,
                                           ip]
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
        lib.vet_model_create.argtypes = [ctypes.POINTER(vp), i, i]
        lib.vet_model_destroy.argtypes = [vp]
        lib.vet_model_num_params.argtypes = [vp]
        lib.vet_model_num_params.restype = ctypes.c_longlong
        for name in ("vet_model_set_params", "vet_model_get_params", "vet_model_get_grads"):
            getattr(lib, name).argtypes = [vp, vp]
        lib.vet_model_features.argtypes = [vp, ctypes.POINTER(_Grid), i, vp, vp, vp, vp, vp]
        lib.vet_model_forward.argtypes = [vp, vp, vp]
        lib.vet_model_backward.argtypes = [vp, vp, vp, ctypes.c_float, vp, vp]
        f = ctypes.c_float
        lib.vet_model_step.argtypes = [vp, f, f, f, f, f, vp]
        lib.vet_closure_learned.argtypes = [vp, vp, vp, vp, vp, vp, f, vp, vp, ip, vp]
        lib.vet_model_last_timing.argtypes = [vp, ctypes.POINTER(f)]
        lib.vet_model_last_indicator.argtypes = [vp, vp, vp]
        lib.vet_hlle_wavespeed.argtypes = [ctypes.POINTER(_Grid), vp, vp, ctypes.c_double, i, vp, vp]
        lib.vet_model_save.argtypes = [vp, ctypes.c_char_p]
        lib.vet_model_load.argtypes = [vp, ctypes.c_char_p]
        lib.vet_model_last_error.argtypes = [vp]
        lib.vet_model_last_error.restype = ctypes.c_char_p
        lib.vet_local_closure.argtypes = [i, ctypes.c_longlong, vp, vp, vp]
        lib.vet_point_source.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                                         vp, vp, vp, vp]
        lib.vet_field_change.argtypes = [ctypes.POINTER(_Grid), vp, vp, vp, vp, i, vp, vp]
        for name in EXPORTS:
            if name not in _NOT_STATUS:
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
        want = {np.float32: torch.float32, np.float64: torch.float64, np.uint8: torch.uint8,
                np.int32: torch.int32}[dtype]
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
        self.block = int(block)
        self.h = float(h)
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

    def moments(self, I, M_out, stream=None, E64_out=None):
        """vet_moments: I [N][cells] -> M_out [10][cells]; E64_out (FP32
        contexts, optional, a float64 CUDA tensor [cells]) receives E summed
        in FP64."""
        nc, dt = self.ncell, self.dtype
        if self.precision == VET_FP64:
            if E64_out is not None:
                raise ValueError("E64_out is for FP32 contexts (the FP64 moments are already double)")
            self._check(self._lib.vet_moments_f64(self._h, _ptr(I, dt, self.N * nc, "I"),
                                                  _ptr(M_out, dt, 10 * nc, "M_out"), _stream(stream)))
        else:
            self._check(self._lib.vet_moments(self._h, _ptr(I, dt, self.N * nc, "I"), _ptr(M_out, dt, 10 * nc, "M_out"),
                                              _ptr(E64_out, np.float64, nc, "E64_out"), _stream(stream)))
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


VET_CLOSURE_EDDINGTON, VET_CLOSURE_M1 = 0, 1


def local_closure(kind: int, M, T_out, ncell: int | None = None, stream=None):
    """vet_local_closure: the Eddington (T = I/3) or M1 tensor of every cell
    from its moments M [10][ncell] into T_out [6][ncell] (device tensors;
    M may be None for the Eddington closure)."""
    lib = load()
    if ncell is None:
        ncell = T_out.numel() // 6
    st = lib.vet_local_closure(int(kind), int(ncell), _ptr(M, np.float32, 10 * ncell, "M"),
                               _ptr(T_out, np.float32, 6 * ncell, "T_out"), _stream(stream))
    if st != VET_OK:
        raise VetError(st, "vet_local_closure")
    return T_out


def point_source(shape, h: float, xs, L: float, kappa, Edot_out, pdot_out=None, stream=None):
    """vet_point_source: energy (Edot_out [cells]) and momentum (pdot_out
    [3][cells], optional) deposition rates of a point source of luminosity L
    at xs (length units) in a grid of `shape` = (nz, ny, nx) cells of edge h;
    kappa [nz][ny][nx] is the opacity to the direct radiation (device)."""
    lib = load()
    nz, ny, nx = shape
    n = int(nz) * int(ny) * int(nx)
    g = _Grid(int(nx), int(ny), int(nz), 1, float(h))
    x = (ctypes.c_double * 3)(*[float(v) for v in xs])
    st = lib.vet_point_source(ctypes.byref(g), x, float(L), _ptr(kappa, np.float32, n, "kappa"),
                              _ptr(Edot_out, np.float32, n, "Edot_out"), _ptr(pdot_out, np.float32, 3 * n, "pdot_out"),
                              _stream(stream))
    if st != VET_OK:
        raise VetError(st, "vet_point_source")
    return Edot_out


def field_change(shape, block: int, h: float, kappa, S, kappa_ref, S_ref, out, snapshot: bool = False,
                 stream=None):
    """vet_field_change: per block of block^3 cells and over the grid, the
    largest bound on the change of a cell's transmission, |a - b| / ((1 +
    a/2)(1 + b/2)) with a = kappa h and b = kappa_ref h, the largest change of
    the source |S - S_ref| and the source scale max |S_ref| (FP32; out [3 + 3
    * blocks], the grid's triple first, blocks x-fastest).  With snapshot the
    same pass copies kappa, S into kappa_ref, S_ref.  Device tensors."""
    lib = load()
    nz, ny, nx = shape
    n = int(nz) * int(ny) * int(nx)
    B = int(block)
    nb = n // (B * B * B) if B > 0 else 0
    g = _Grid(int(nx), int(ny), int(nz), B, float(h))
    st = lib.vet_field_change(ctypes.byref(g), _ptr(kappa, np.float32, n, "kappa"), _ptr(S, np.float32, n, "S"),
                              _ptr(kappa_ref, np.float32, n, "kappa_ref"), _ptr(S_ref, np.float32, n, "S_ref"),
                              int(bool(snapshot)), _ptr(out, np.float32, 3 + 3 * nb, "out"), _stream(stream))
    if st != VET_OK:
        raise VetError(st, "vet_field_change")
    return out


def hlle_wavespeed(shape, h: float, f, kappa_R, C_out, axis: int, c: float = 1.0, stream=None):
    """vet_hlle_wavespeed: corrected HLLE wavespeeds of the faces normal to
    `axis` (0 = x) of a grid of `shape` = (nz, ny, nx) cells of edge h, from
    f [6][cells] and kappa_R [cells] (device); C_out has one more point along
    the axis (see include/vet.h)."""
    lib = load()
    nz, ny, nx = (int(v) for v in shape)
    n = nz * ny * nx
    ext = [nz, ny, nx]
    ext[2 - int(axis)] += 1
    g = _Grid(nx, ny, nz, 1, float(h))
    st = lib.vet_hlle_wavespeed(ctypes.byref(g), _ptr(f, np.float32, 6 * n, "f"), _ptr(kappa_R, np.float32, n, "kappa_R"),
                                float(c), int(axis), _ptr(C_out, np.float32, int(np.prod(ext)), "C_out"),
                                _stream(stream))
    if st != VET_OK:
        raise VetError(st, "vet_hlle_wavespeed")
    return C_out


def reuse_decision(change, age: int, first: bool, tol_tau: float, tol_S: float, max_age: int) -> bool:
    """Whether a stored Eddington tensor must be recomputed this time step
    (paper Sec. 4.2): always on the first step and once it is max_age steps
    old; otherwise when the grid's largest transmission change exceeds
    tol_tau or its largest source change exceeds tol_S times the source
    scale.  `change` is the grid triple (dtrans, dS, Sref) of field_change;
    a non-finite change forces a recompute."""
    lib = load()
    c = (ctypes.c_float * 3)(*[float(v) for v in change[:3]])
    out = ctypes.c_int()
    st = lib.vet_reuse_decision(c, int(age), int(bool(first)), float(tol_tau), float(tol_S), int(max_age),
                                ctypes.byref(out))
    if st != VET_OK:
        raise VetError(st, "vet_reuse_decision: bad age, max_age or tolerance")
    return bool(out.value)


class ClosureReuse:
    """Time steps of the closure that reuse f while its inputs stay close to
    the snapshot f was computed from (paper Sec. 4.2's suggestion of updating
    the Eddington tensor only every few steps).  Each step runs the change
    gate (vet_field_change) against the snapshot, reads the grid's three
    numbers back to the host (12 bytes; the step synchronises the stream),
    and either keeps the stored f or recomputes it with the context and takes
    a new snapshot.  Owns the snapshot and f (device, FP32).

    The boundary intensities are not watched: pass force=True on a step
    whose Ib differs from the one f was computed with."""

    def __init__(self, ctx: Context, tol_tau: float = 5e-2, tol_S: float = 5e-2, max_age: int = 8):
        import torch

        if ctx.precision != VET_FP32:
            raise ValueError("ClosureReuse needs an FP32 context")
        if max_age < 1:
            raise ValueError("max_age must be at least 1")
        self.ctx, self.tol_tau, self.tol_S, self.max_age = ctx, float(tol_tau), float(tol_S), int(max_age)
        dev = torch.device("cuda", torch.cuda.current_device())
        n, B = ctx.ncell, ctx.block
        self.kappa_ref = torch.zeros(n, dtype=torch.float32, device=dev)
        self.S_ref = torch.zeros(n, dtype=torch.float32, device=dev)
        self.change = torch.zeros(3 + 3 * (n // (B * B * B)), dtype=torch.float32, device=dev)
        self._host = torch.zeros(3, dtype=torch.float32).pin_memory()
        self.f = torch.zeros(6 * n, dtype=torch.float32, device=dev)
        self.age, self.first = 0, True
        self.recomputes = 0
        self.last_change = (0.0, 0.0, 0.0)

    def step(self, kappa, S, Ib=None, M_out=None, force: bool = False, stream=None):
        """One time step: returns (f, recomputed).  M_out, if given, is
        written only on steps that recompute."""
        import torch

        st = _stream(stream)
        if not self.first:
            field_change(self.ctx.shape, self.ctx.block, self.ctx.h, kappa, S, self.kappa_ref, self.S_ref,
                         self.change, False, st)
            s = torch.cuda.ExternalStream(st) if st else torch.cuda.current_stream()
            with torch.cuda.stream(s):
                self._host.copy_(self.change[:3], non_blocking=True)
            s.synchronize()
            self.last_change = tuple(float(v) for v in self._host)
        redo = force or reuse_decision(self.last_change, self.age, self.first, self.tol_tau, self.tol_S,
                                       self.max_age)
        if redo:
            self.ctx.closure(kappa, S, Ib, self.f, M_out, stream=st)
            field_change(self.ctx.shape, self.ctx.block, self.ctx.h, kappa, S, self.kappa_ref, self.S_ref,
                         self.change, True, st)
            self.age, self.first = 0, False
            self.recomputes += 1
        else:
            self.age += 1
        return self.f, redo


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

    def __init__(self, lib, handle, shape, block):
        self._lib = lib
        self._h = ctypes.c_void_p(handle)
        self.shape = tuple(int(v) for v in shape)
        self.block = int(block)
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
        self.members = [_Member(self._lib, self._lib.vet_batch_context(self._h, i), problems[i][0], problems[i][1])
                        for i in range(n)]

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


#: (input, output) channels of the four convolutions for `channels` hidden channels
def layer_shapes(channels: int = 32):
    return [(6, channels), (channels, channels), (channels, channels), (channels, 7)]


class Model:
    """vet_model: the learned closure's network, its optimiser state and
    workspace (include/vet.h).  Parameters cross as a list of (W, b) with
    W[27][C_out][C_in] and b[C_out] per layer."""

    def __init__(self, channels: int = 32, device: int = 0):
        self._lib = load()
        h_ = ctypes.c_void_p()
        st = self._lib.vet_model_create(ctypes.byref(h_), int(channels), int(device))
        if st != VET_OK:
            raise VetError(st, self._lib.vet_model_last_error(None).decode())
        self._h = h_
        self.channels = int(channels)
        self.shapes = layer_shapes(self.channels)
        self.num_params = int(self._lib.vet_model_num_params(self._h))
        self.nvol = 0
        self.ncell = 0

    def close(self):
        if getattr(self, "_h", None):
            self._lib.vet_model_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != VET_OK:
            raise VetError(st, self._lib.vet_model_last_error(self._h).decode())

    def _flat(self, params):
        parts = []
        for (W, b), (ci, co) in zip(params, self.shapes):
            W = np.asarray(W, dtype=np.float32)
            b = np.asarray(b, dtype=np.float32)
            if W.shape != (27, co, ci) or b.shape != (co,):
                raise ValueError(f"layer shapes: expected W {(27, co, ci)}, b {(co,)}; got {W.shape}, {b.shape}")
            parts += [W.ravel(), b.ravel()]
        flat = np.ascontiguousarray(np.concatenate(parts))
        assert flat.size == self.num_params
        return flat

    def _unflat(self, flat):
        out, k = [], 0
        for ci, co in self.shapes:
            W = flat[k:k + 27 * co * ci].reshape(27, co, ci)
            k += 27 * co * ci
            b = flat[k:k + co]
            k += co
            out.append((W.copy(), b.copy()))
        return out

    def set_params(self, params):
        flat = self._flat(params)
        self._check(self._lib.vet_model_set_params(self._h, flat.ctypes.data))

    def params(self):
        flat = np.zeros(self.num_params, dtype=np.float32)
        self._check(self._lib.vet_model_get_params(self._h, flat.ctypes.data))
        return self._unflat(flat)

    def grads(self):
        flat = np.zeros(self.num_params, dtype=np.float32)
        self._check(self._lib.vet_model_get_grads(self._h, flat.ctypes.data))
        return self._unflat(flat)

    def save(self, path):
        """vet_model_save: parameters, AdamW state and step count to a file."""
        self._check(self._lib.vet_model_save(self._h, os.fsencode(os.fspath(path))))

    def load(self, path):
        """vet_model_load: read a file written by save() (the hidden width
        and parameter count must match)."""
        self._check(self._lib.vet_model_load(self._h, os.fsencode(os.fspath(path))))

    def features(self, shape, block: int, h: float, kappa, S, E, nvol: int = 1, feat_out=None, stream=None):
        """Features of nvol stacked volumes of `shape` (device tensors)."""
        nz, ny, nx = (int(v) for v in shape)
        n = nvol * nz * ny * nx
        g = _Grid(nx, ny, nz, int(block), float(h))
        self._check(self._lib.vet_model_features(
            self._h, ctypes.byref(g), int(nvol), _ptr(kappa, np.float32, n, "kappa"), _ptr(S, np.float32, n, "S"),
            _ptr(E, np.float32, n, "E"), _ptr(feat_out, np.float32, 6 * n, "feat_out"), _stream(stream)))
        self.nvol, self.ncell = int(nvol), n
        return feat_out

    def forward(self, o_out=None, stream=None):
        self._check(self._lib.vet_model_forward(self._h, _ptr(o_out, np.float32, 7 * self.ncell, "o_out"),
                                                _stream(stream)))
        return o_out

    def backward(self, f_ref, mask=None, lam: float = 0.01, loss_out=None, stream=None):
        n = self.ncell
        self._check(self._lib.vet_model_backward(self._h, _ptr(f_ref, np.float32, 6 * n, "f_ref"),
                                                 _ptr(mask, np.uint8, n, "mask"), float(lam),
                                                 _ptr(loss_out, np.float64, 1, "loss_out"), _stream(stream)))
        return loss_out

    def step(self, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
             weight_decay: float = 1e-4, stream=None):
        self._check(self._lib.vet_model_step(self._h, float(lr), float(beta1), float(beta2), float(eps),
                                             float(weight_decay), _stream(stream)))

    def closure(self, ctx: Context, kappa, S, E, f_out, Ib=None, threshold: float = 1e-2, block_flags=None,
                stream=None) -> int:
        """vet_closure_learned on ctx's grid; returns the number of blocks
        recomputed by the exact closure."""
        nc = ctx.ncell
        nfb = ctypes.c_int(0)
        nblk = nc // (ctx.block ** 3)
        st = self._lib.vet_closure_learned(
            ctx._h, self._h, _ptr(kappa, np.float32, nc, "kappa"), _ptr(S, np.float32, nc, "S"),
            _ptr(E, np.float32, nc, "E"), _ptr(Ib, np.float32, 6 * ctx.N, "Ib"), float(threshold),
            _ptr(f_out, np.float32, 6 * nc, "f_out"), _ptr(block_flags, np.int32, nblk, "block_flags"),
            ctypes.byref(nfb), _stream(stream))
        self._check(st)
        return nfb.value

    def last_timing(self):
        """(network, fallback, whole call, convolutions) in ms of the last
        learned closure."""
        ms = (ctypes.c_float * 4)()
        self._check(self._lib.vet_model_last_timing(self._h, ms))
        return tuple(float(v) for v in ms)

    def last_indicator(self, r_out, ncell: int, stream=None):
        self._check(self._lib.vet_model_last_indicator(self._h, _ptr(r_out, np.float32, ncell, "r_out"),
                                                       _stream(stream)))
        return r_out
