"""FP64 oracle of the two local closures the paper compares the VET with
(Sec. 4.1, "Comparison to FLD and M1 schemes").

TEST INFRASTRUCTURE: imported only by the tests and the benchmark's CPU
baseline; it shares nothing with the product library.

Both map the moments of one cell to an Eddington tensor, cell by cell:
  eddington -- T = I / 3 (the paper's stand-in for FLD);
  m1        -- T = (1 - chi)/2 I + (3 chi - 1)/2 n n, n = F / |F|, with
               chi(f) = (3 + 4 f^2) / (5 + 2 sqrt(4 - 3 f^2)), f = |F| / (c E)
               and c = 1 (the moments here carry no factor c).
Readings where the paper is silent: f is clipped to [0, 1] (a flux above
c E is unphysical and chi is not real beyond f = 4/3); F = 0 leaves chi =
1/3, where the n n term vanishes whatever n; E <= 0 gives T = I / 3 (the
fallback the VET closure uses).  The plain loop below restates the formulas
one cell at a time; it is slow and meant for test-sized inputs.

Layout: M [10][cells] = (E, Fx, Fy, Fz, Pxx, Pyy, Pzz, Pxy, Pxz, Pyz) (only
E and F are read); T [6][cells] = (xx, yy, zz, xy, xz, yz).
"""
from __future__ import annotations

import math

import numpy as np


def chi(f: float) -> float:
    """The M1 Eddington factor of a reduced flux f in [0, 1]."""
    return (3.0 + 4.0 * f * f) / (5.0 + 2.0 * math.sqrt(4.0 - 3.0 * f * f))


def eddington(ncell: int) -> np.ndarray:
    T = np.zeros((6, ncell))
    T[:3] = 1.0 / 3.0
    return T


def m1(M) -> np.ndarray:
    M = np.asarray(M, dtype=np.float64).reshape(10, -1)
    n = M.shape[1]
    T = np.zeros((6, n))
    for c in range(n):
        E, Fx, Fy, Fz = M[0, c], M[1, c], M[2, c], M[3, c]
        if not E > 0.0:
            T[:3, c] = 1.0 / 3.0
            continue
        Fn = math.sqrt(Fx * Fx + Fy * Fy + Fz * Fz)
        f = min(Fn / E, 1.0)
        x = chi(f)
        a, b = (1.0 - x) / 2.0, (3.0 * x - 1.0) / 2.0
        if Fn > 0.0:
            nx, ny, nz = Fx / Fn, Fy / Fn, Fz / Fn
        else:
            nx = ny = nz = 0.0  # b = 0 here: chi(0) = 1/3
        T[0, c] = a + b * nx * nx
        T[1, c] = a + b * ny * ny
        T[2, c] = a + b * nz * nz
        T[3, c] = b * nx * ny
        T[4, c] = b * nx * nz
        T[5, c] = b * ny * nz
    return T
