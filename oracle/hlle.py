"""FP64 oracle of the HLLE face wavespeed with the optical-depth correction
(Sec. 2.2.3, "Implicit Hyperbolic Transport of Radiation", and App. A), the
first consumer of the Eddington tensor f.

TEST INFRASTRUCTURE: imported only by the tests and the benchmark's CPU
baseline; it shares nothing with the product library.

The paper's wavespeed of the radiation subsystem across a face normal to
axis a is the free-streaming eigenvalue sqrt(f_aa) c of the moment
equations times the correction factor sqrt((1 - e^-tau_c) / tau_c), with
tau_c = (10 dl rho kappa_R)^2 / (2 f_aa) (dl the cell thickness, f_aa the
diagonal component of f along the flux), taken at an interface between two
cells of one refinement level as the arithmetic mean of the two cells'
values.  Readings where the paper is silent (a uniform grid has no level
jumps, so the upstream rule of level boundaries does not arise):
  - each cell's tau is formed with that cell's own f_aa and kappa_R;
  - the free-streaming factor of a face is the larger of the two cells'
    sqrt(f_aa) (the usual HLLE bound on the fastest wave of either state);
    the left- and right-going speeds are minus and plus the returned value;
  - a face on the domain boundary has one cell, whose values it takes;
  - f_aa <= 0 gives tau = +inf, so the cell's factor sqrt(f_aa) g(tau) is
    0 (its limit as f_aa -> 0 at fixed kappa); kappa_R = 0 gives tau = 0
    and g = 1; g(tau) = sqrt(-expm1(-tau) / tau).
The plain loops below restate the formulas one face at a time; they are slow
and meant for test-sized inputs.

Layout: f [6][nz][ny][nx] (xx, yy, zz, xy, xz, yz), kappa_R [nz][ny][nx]
(rho kappa_R per unit length), cell thickness h; the faces normal to axis a
(0 = x) are the grid with one more point along a: C [nz][ny][nx + 1] for
a = 0, [nz][ny + 1][nx] for a = 1, [nz + 1][ny][nx] for a = 2.
"""
from __future__ import annotations

import math

import numpy as np


def cell_tau(f_aa: float, kappa: float, h: float) -> float:
    """tau_c of one cell: (10 h kappa)^2 / (2 f_aa)."""
    if f_aa <= 0.0:
        return math.inf
    return (10.0 * h * kappa) ** 2 / (2.0 * f_aa)


def correction(tau: float) -> float:
    """sqrt((1 - e^-tau) / tau), 1 at tau = 0 and 0 at tau = inf."""
    if tau == 0.0:
        return 1.0
    if math.isinf(tau):
        return 0.0
    return math.sqrt(-math.expm1(-tau) / tau)


def face_speed(fL: float, kL: float, fR: float, kR: float, h: float, c: float = 1.0) -> float:
    """Wavespeed magnitude at a face between cells L and R of one level."""
    tau = 0.5 * (cell_tau(fL, kL, h) + cell_tau(fR, kR, h))
    s = math.sqrt(max(fL, fR, 0.0))
    if s == 0.0:
        return 0.0
    return s * c * correction(tau)


def wavespeeds(f, kappa_R, h: float, axis: int, c: float = 1.0) -> np.ndarray:
    """Face wavespeeds of the whole grid along `axis` (see the layout above)."""
    f = np.asarray(f, dtype=np.float64)
    k = np.asarray(kappa_R, dtype=np.float64)
    nz, ny, nx = k.shape
    faa = f[axis].reshape(nz, ny, nx)
    shape = [nz, ny, nx]
    shape[2 - axis] += 1
    out = np.empty(shape)
    for iz in range(shape[0]):
        for iy in range(shape[1]):
            for ix in range(shape[2]):
                idx = [iz, iy, ix]
                lo = list(idx)
                lo[2 - axis] -= 1  # the cell on the low side of the face
                hi = idx
                n_along = (nz, ny, nx)[2 - axis]
                have_lo = lo[2 - axis] >= 0
                have_hi = hi[2 - axis] < n_along
                if have_lo and have_hi:
                    out[iz, iy, ix] = face_speed(faa[tuple(lo)], k[tuple(lo)], faa[tuple(hi)], k[tuple(hi)], h, c)
                else:
                    cell = tuple(lo) if have_lo else tuple(hi)
                    out[iz, iy, ix] = face_speed(faa[cell], k[cell], faa[cell], k[cell], h, c)
    return out
