"""FP64 oracle of the point-source contribution (paper Sec. 2.2.6, "Point
Sources Contribution"): the energy and momentum a point source deposits in
every cell through the direct radiation.

TEST INFRASTRUCTURE: imported only by the tests and the benchmark's CPU
baseline; it shares nothing with the product library.

For every cell c the straight ray from the source position x_s through the
cell centre x_c is followed (long characteristics, the limit the paper's
hybrid tracer approximates):
  tau_*    optical depth sum kappa * length over the cells the ray crosses
           from x_s to where it enters c (0 if the source lies in c);
  dr       length of the ray inside c, from where it enters c (or from x_s
           if the source lies in c) to where it leaves c;
  tau_cell kappa_c * dr;
  Edot     L e^{-tau_*} (1 - e^{-tau_cell}) / (4 pi r^2 dr), r = |x_c - x_s|,
           with 1 - e^{-tau_cell} evaluated as -expm1(-tau_cell), which is
           the paper's Taylor form tau_cell for small tau_cell without a
           switch;
  pdot     Edot / c * (x_c - x_s) / r with c = 1.
Readings: cells are [i, i+1) h per axis; a ray point on a cell face lies in
the cell the ray enters next; a cell whose centre coincides with the source
(r = 0) gets Edot = pdot = 0.

Layout: kappa [nz][ny][nx] (per unit length); Edot [cells]; pdot [3][cells].
"""
from __future__ import annotations

import math

import numpy as np


def _cell_range(x0, d, lo, hi):
    """Parameter interval [t_in, t_out] of the line x0 + t d inside the box
    [lo, hi) (slab intersection)."""
    t_in, t_out = -math.inf, math.inf
    for a in range(3):
        if d[a] != 0.0:
            t1 = (lo[a] - x0[a]) / d[a]
            t2 = (hi[a] - x0[a]) / d[a]
            t_in = max(t_in, min(t1, t2))
            t_out = min(t_out, max(t1, t2))
        elif not (lo[a] <= x0[a] < hi[a]):
            return math.inf, -math.inf
    return t_in, t_out


def optical_depth(kappa, h, xs, xc, nsteps=None):
    """tau_* and dr for the ray from xs through the centre xc (FP64 DDA in
    cell units: the crossings of the planes x = m h along each axis are
    merged in order)."""
    nz, ny, nx = kappa.shape
    dvec = np.asarray(xc, float) - np.asarray(xs, float)
    r = math.sqrt(float(dvec @ dvec))
    d = dvec / r  # unit direction; parameter t = distance from xs
    ci = [int(math.floor(xc[0] / h)), int(math.floor(xc[1] / h)), int(math.floor(xc[2] / h))]
    lo = [ci[a] * h for a in range(3)]
    hi = [(ci[a] + 1) * h for a in range(3)]
    t_in, t_out = _cell_range(xs, d, lo, hi)
    t_in = max(t_in, 0.0)
    dr = t_out - t_in
    # cells from the source up to the entry of the target cell
    tau = 0.0
    cur = [int(math.floor(xs[a] / h)) for a in range(3)]
    t = 0.0
    dims = (nx, ny, nz)
    while t < t_in - 1e-12 * h:
        # next plane crossing
        t_next, ax = math.inf, -1
        for a in range(3):
            if d[a] > 0.0:
                tp = ((cur[a] + 1) * h - xs[a]) / d[a]
            elif d[a] < 0.0:
                tp = (cur[a] * h - xs[a]) / d[a]
            else:
                continue
            if tp < t_next:
                t_next, ax = tp, a
        t_next = min(t_next, t_in)
        if 0 <= cur[0] < dims[0] and 0 <= cur[1] < dims[1] and 0 <= cur[2] < dims[2]:
            tau += kappa[cur[2], cur[1], cur[0]] * (t_next - t)
        t = t_next
        if t >= t_in - 1e-12 * h:
            break
        cur[ax] += 1 if d[ax] > 0.0 else -1
    return tau, dr, r, d


def deposit(kappa, h, xs, L):
    """Edot [cells] and pdot [3][cells] of a source of luminosity L at xs."""
    kappa = np.asarray(kappa, dtype=np.float64)
    nz, ny, nx = kappa.shape
    Edot = np.zeros(kappa.size)
    pdot = np.zeros((3, kappa.size))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                c = (k * ny + j) * nx + i
                xc = ((i + 0.5) * h, (j + 0.5) * h, (k + 0.5) * h)
                if all(abs(xc[a] - xs[a]) == 0.0 for a in range(3)):
                    continue
                tau, dr, r, d = optical_depth(kappa, h, xs, xc)
                tc = kappa[k, j, i] * dr
                e = L * math.exp(-tau) * (-math.expm1(-tc)) / (4.0 * math.pi * r * r * dr)
                Edot[c] = e
                pdot[:, c] = e * d
    return Edot, pdot
