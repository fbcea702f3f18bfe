"""Pins of the point-source oracle (oracle/point_source.py; paper Sec.
2.2.6): the optical depth and the in-cell path against brute-force sampling
of the ray, the vacuum and small-tau (Taylor) limits, the momentum
direction, and mirror symmetry."""
import math

import numpy as np

from oracle import point_source as ps


def _brute(kappa, h, xs, xc, n=200000):
    """tau_* and dr by sampling the segment xs -> xc (and beyond, for dr) at
    n points per ray length: the cell of each midpoint decides."""
    nz, ny, nx = kappa.shape
    xs, xc = np.asarray(xs, float), np.asarray(xc, float)
    r = np.linalg.norm(xc - xs)
    d = (xc - xs) / r
    span = r + 2.0 * math.sqrt(3.0) * h
    t = (np.arange(n) + 0.5) * (span / n)
    p = xs[None, :] + t[:, None] * d[None, :]
    idx = np.floor(p / h).astype(int)
    tgt = np.floor(xc / h).astype(int)
    inside = np.all(idx == tgt[None, :], axis=1)
    ok = np.all((idx >= 0) & (idx < np.array([nx, ny, nz])), axis=1)
    first = np.argmax(inside)
    kap = np.where(ok, kappa[np.clip(idx[:, 2], 0, nz - 1), np.clip(idx[:, 1], 0, ny - 1),
                             np.clip(idx[:, 0], 0, nx - 1)], 0.0)
    ds = span / n
    tau = kap[:first].sum() * ds
    dr = inside.sum() * ds
    return tau, dr


def test_depth_and_path_against_sampling():
    rng = np.random.default_rng(3)
    kappa = rng.lognormal(0.0, 1.0, (6, 7, 8))
    h = 0.25
    xs = (0.9, 1.1, 0.35)
    for c in rng.choice(kappa.size, 12, replace=False):
        k, j, i = np.unravel_index(c, kappa.shape)
        xc = ((i + 0.5) * h, (j + 0.5) * h, (k + 0.5) * h)
        tau, dr, r, d = ps.optical_depth(kappa, h, xs, xc)
        tb, db = _brute(kappa, h, xs, xc)
        assert abs(tau - tb) < 2e-4 * (1.0 + tau), (tau, tb)
        assert abs(dr - db) < 2e-4 * h, (dr, db)
        assert abs(r - math.dist(xs, xc)) < 1e-12


def test_vacuum_deposits_nothing_and_thin_cells_take_the_taylor_form():
    h, L, xs = 0.1, 3.0, (0.4, 0.4, 0.4)  # a lattice point
    E0, p0 = ps.deposit(np.zeros((8, 8, 8)), h, xs, L)
    assert np.all(E0 == 0.0) and np.all(p0 == 0.0)
    kap = 1e-6
    E, p = ps.deposit(np.full((8, 8, 8), kap), h, xs, L)
    Z, Y, X = np.meshgrid(*(((np.arange(8) + 0.5) * h),) * 3, indexing="ij")
    r2 = ((X - xs[0]) ** 2 + (Y - xs[1]) ** 2 + (Z - xs[2]) ** 2).ravel()
    taylor = kap * L / (4.0 * math.pi * r2)   # the paper's small-tau form, e^{-tau_*} ~ 1
    np.testing.assert_allclose(E, taylor, rtol=5e-6)


def test_momentum_points_away_from_the_source_with_magnitude_edot():
    rng = np.random.default_rng(4)
    kappa = rng.uniform(0.5, 2.0, (5, 5, 5))
    h, xs = 0.2, (0.31, 0.52, 0.47)
    E, p = ps.deposit(kappa, h, xs, 1.0)
    Z, Y, X = np.meshgrid(*(((np.arange(5) + 0.5) * h),) * 3, indexing="ij")
    v = np.stack([X.ravel() - xs[0], Y.ravel() - xs[1], Z.ravel() - xs[2]])
    v /= np.linalg.norm(v, axis=0)
    np.testing.assert_allclose(p, E[None, :] * v, rtol=1e-12, atol=1e-300)
    assert np.all(E > 0)


def test_mirror_symmetry_about_a_central_source():
    kappa = np.full((6, 6, 6), 1.5)
    kappa[:, :, :3] = 0.7  # symmetric under y and z reflections only
    h, xs = 0.5, (1.5, 1.5, 1.5)
    E, _ = ps.deposit(kappa, h, xs, 2.0)
    E = E.reshape(6, 6, 6)
    np.testing.assert_allclose(E, E[::-1, :, :], rtol=1e-12)   # z -> -z
    np.testing.assert_allclose(E, E[:, ::-1, :], rtol=1e-12)   # y -> -y
