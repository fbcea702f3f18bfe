"""ctypes front end of the FP64 C oracle (``vet_oracle.c``).

TEST INFRASTRUCTURE: imported only by the tests, the smoke check and the
CPU-baseline leg of the benchmark.  It holds no CUDA code and shares nothing
with the product library.

Functions follow the paper's steps (VETTAM, Sec. 2.2.5):
  healpix   -- HEALPix direction set, equal weights 4 pi / N, rotated;
  trace     -- hybrid-characteristics formal solution of Eq. 14 (RTeq);
  moments   -- E, F_i, P_ij quadratures (Eqs. 10-12, c = 1);
  closure   -- f_ij = P_ij / E (Eq. 13) with the isotropic fallback where E
               does not exceed floor_rel * max E.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vet_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libvet_oracle.so")
_lib = None
_lock = threading.Lock()


class _Grid(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("nz", ctypes.c_int),
        ("B", ctypes.c_int),
        ("h", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -O2) into oracle/_build."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"],
            check=True,
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.ora_healpix.argtypes = [ctypes.c_int, dp, dp]
            lib.ora_trace.argtypes = [ctypes.POINTER(_Grid), dp, ctypes.c_int, dp, dp, dp, dp, ctypes.c_int]
            lib.ora_moments.argtypes = [dp, dp, ctypes.c_int, ctypes.c_long, dp]
            lib.ora_closure.argtypes = [dp, ctypes.c_long, ctypes.c_double, dp, ctypes.POINTER(ctypes.c_ubyte)]
            lib.ora_count_segments.argtypes = [ctypes.POINTER(_Grid), dp, ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_longlong)]
            lib.ora_count_segments.restype = ctypes.c_longlong
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def healpix(nside: int, q=None) -> np.ndarray:
    """[N][4] directions (nx, ny, nz, w); q = unit quaternion (w, x, y, z) or None."""
    lib = _load()
    n = 12 * nside * nside
    out = np.zeros((n, 4), dtype=np.float64)
    qa = None if q is None else _f64(q)
    st = lib.ora_healpix(nside, None if qa is None else _dp(qa), _dp(out))
    if st != 0:
        raise ValueError(f"ora_healpix failed ({st}) for nside={nside}")
    return out


def _grid(shape, B: int, h: float) -> _Grid:
    nz, ny, nx = shape
    return _Grid(nx, ny, nz, B, h)


def trace(kappa, S, dirs, B: int, h: float, Ib=None, nthreads: int | None = None) -> np.ndarray:
    """Cell-centre intensities I [ndir][nz][ny][nx] for every direction.

    kappa, S: [nz][ny][nx]; dirs: [ndir][4]; Ib: [6][ndir] or None (vacuum)."""
    lib = _load()
    kappa = _f64(kappa)
    S = _f64(S)
    dirs = _f64(dirs)
    if kappa.ndim != 3 or kappa.shape != S.shape:
        raise ValueError("kappa and S must be 3-D arrays of one shape")
    ndir = dirs.shape[0]
    Iba = None if Ib is None else _f64(Ib)
    if Iba is not None and Iba.shape != (6, ndir):
        raise ValueError("Ib must be [6][ndir]")
    out = np.empty((ndir,) + kappa.shape, dtype=np.float64)
    g = _grid(kappa.shape, B, h)
    if nthreads is None:
        nthreads = max(1, len(os.sched_getaffinity(0)))
    st = lib.ora_trace(ctypes.byref(g), _dp(dirs), ndir, _dp(kappa), _dp(S),
                       None if Iba is None else _dp(Iba), _dp(out), int(nthreads))
    if st != 0:
        raise ValueError(f"ora_trace failed ({st})")
    return out


def moments(I, dirs) -> np.ndarray:
    """M [10][cells...] = E, Fx, Fy, Fz, Pxx, Pyy, Pzz, Pxy, Pxz, Pyz."""
    lib = _load()
    I = _f64(I)
    dirs = _f64(dirs)
    ndir = dirs.shape[0]
    cell_shape = I.shape[1:]
    ncell = int(np.prod(cell_shape))
    out = np.empty((10,) + cell_shape, dtype=np.float64)
    st = lib.ora_moments(_dp(I), _dp(dirs), ndir, ncell, _dp(out))
    if st != 0:
        raise ValueError(f"ora_moments failed ({st})")
    return out


def closure(M, floor_rel: float = 1e-30):
    """(f [6][cells...] = xx, yy, zz, xy, xz, yz;  iso flag [cells...])."""
    lib = _load()
    M = _f64(M)
    cell_shape = M.shape[1:]
    ncell = int(np.prod(cell_shape))
    f = np.empty((6,) + cell_shape, dtype=np.float64)
    flag = np.zeros(cell_shape, dtype=np.uint8)
    st = lib.ora_closure(_dp(M), ncell, float(floor_rel), _dp(f),
                         flag.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
    if st != 0:
        raise ValueError(f"ora_closure failed ({st})")
    return f, flag


def vet_closure(kappa, S, dirs, B: int, h: float, Ib=None, nthreads=None, floor_rel=1e-30):
    """Whole path: trace -> moments -> closure.  Returns (f, M, I, iso)."""
    I = trace(kappa, S, dirs, B, h, Ib, nthreads)
    M = moments(I, dirs)
    f, iso = closure(M, floor_rel)
    return f, M, I, iso


def count_segments(shape, B: int, dirs):
    """(cell-ray segments, face-node-ray segments) summed over the grid's
    blocks and the given directions: the work measure of the method."""
    lib = _load()
    dirs = _f64(dirs)
    g = _grid(shape, B, 1.0)
    face = ctypes.c_longlong(0)
    n = lib.ora_count_segments(ctypes.byref(g), _dp(dirs), dirs.shape[0], ctypes.byref(face))
    if n < 0:
        raise ValueError("ora_count_segments failed")
    return int(n), int(face.value)
