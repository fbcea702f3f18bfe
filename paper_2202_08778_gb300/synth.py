"""Seeded synthetic inputs for the VET closure (opacity, source function,
boundary intensities, direction-set rotation).

This module draws random numbers and lays out test fields; it contains none
of the method's arithmetic (no transfer, no quadrature, no closure), so both
the CUDA path and the CPU oracle can take their inputs from it.

Units: kappa is the absorption coefficient per unit length (rho kappa_P of the
paper), h the cell edge in the same length unit, and the source function is
S = a_R c T^4 / (4 pi) with a_R = c = 1 (VETTAM Sec. 2.1, Eq. 14 text).

Workloads (shapes of the paper's shadow and clump test problems, Sec. 3.8):
  blob_problem      -- uniform kappa = 0.1 plus a Gaussian blob of peak 10 and
                       sigma 0.1 box at the centre; T = 1 + 9 exp(-r^2/0.02);
                       vacuum boundaries (32^3, blocks of 8^3, 48 directions).
  lognormal_problem -- lognormal kappa (sigma_ln = 1.5, P(k) ~ k^-2 on
                       2 <= |k| <= 32, median cell optical depth 10^-0.5,
                       clipped to [1e-3, 1e2]); lognormal T (sigma_ln = 0.5,
                       correlation 0.5 with kappa); vacuum boundaries
                       (128^3, blocks of 16^3, 192 directions).
  cloud_problem     -- 2x1x1 box, ambient kappa = 1e-2, ellipsoidal cloud of
                       kappa = 1e3 with a two-cell tanh edge, S = 0, a beam of
                       I = 1 entering through x = 0 for directions within 10
                       degrees of +x (256x128x128, 16^3 blocks, 768 dirs).
"""
from __future__ import annotations

import math

import numpy as np

FOUR_PI = 4.0 * math.pi


def rotation_quaternion(seed: int) -> np.ndarray:
    """Unit quaternion (w, x, y, z) uniform on S^3 (a Haar-random rotation):
    four standard normals from numpy's PCG64 stream ``seed``, normalised."""
    rng = np.random.default_rng(seed)
    q = rng.standard_normal(4)
    return q / np.linalg.norm(q)


IDENTITY_Q = np.array([1.0, 0.0, 0.0, 0.0])


def _centres(shape, h):
    nz, ny, nx = shape
    z = (np.arange(nz) + 0.5) * h
    y = (np.arange(ny) + 0.5) * h
    x = (np.arange(nx) + 0.5) * h
    return np.meshgrid(z, y, x, indexing="ij")


def gaussian_random_field(shape, rng, kmin=2.0, kmax=32.0, slope=-2.0) -> np.ndarray:
    """Zero-mean, unit-variance Gaussian field with power P(k) ~ k^slope for
    kmin <= |k| <= kmax (integer box wavenumbers of the longest axis' box),
    zero elsewhere; white noise filtered in Fourier space."""
    nz, ny, nx = shape
    L = max(shape)
    white = rng.standard_normal(shape)
    wk = np.fft.rfftn(white)
    kz = np.fft.fftfreq(nz, d=1.0 / nz) * (L / nz)
    ky = np.fft.fftfreq(ny, d=1.0 / ny) * (L / ny)
    kx = np.fft.rfftfreq(nx, d=1.0 / nx) * (L / nx)
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    k = np.sqrt(KZ * KZ + KY * KY + KX * KX)
    kmax = min(kmax, 0.5 * min(shape) * L / max(shape))
    amp = np.zeros_like(k)
    band = (k >= kmin) & (k <= kmax)
    amp[band] = k[band] ** (0.5 * slope)
    g = np.fft.irfftn(wk * amp, s=shape, axes=(0, 1, 2))
    g -= g.mean()
    sd = g.std()
    return g / sd if sd > 0 else g


def blob_problem(n: int = 32, B: int = 8, nside: int = 2, seed: int = 1, rotate: bool = True):
    h = 1.0 / n
    Z, Y, X = _centres((n, n, n), h)
    r2 = (X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2
    kappa = 0.1 + 10.0 * np.exp(-r2 / (2 * 0.1 ** 2))
    T = 1.0 + 9.0 * np.exp(-r2 / 0.02)
    S = T ** 4 / FOUR_PI
    return dict(name=f"blob{n}", kappa=kappa, S=S, B=B, h=h, nside=nside,
                q=rotation_quaternion(seed) if rotate else IDENTITY_Q.copy(), Ib=None)


def lognormal_problem(n: int = 128, B: int = 16, nside: int = 4, seed: int = 2, rotate: bool = True,
                      sigma_ln_kappa: float = 1.5, sigma_ln_T: float = 0.5, rho: float = 0.5,
                      median_dtau: float = 10 ** -0.5, dtau_clip=(1e-3, 1e2), shape=None):
    shape = (n, n, n) if shape is None else tuple(shape)
    h = 1.0 / max(shape)
    rng = np.random.default_rng(seed)
    g1 = gaussian_random_field(shape, rng)
    g2 = gaussian_random_field(shape, rng)
    dtau = np.exp(math.log(median_dtau) + sigma_ln_kappa * g1)
    dtau = np.clip(dtau, dtau_clip[0], dtau_clip[1])
    kappa = dtau / h
    lnT = sigma_ln_T * (rho * g1 + math.sqrt(1.0 - rho * rho) * g2)
    S = np.exp(4.0 * lnT) / FOUR_PI
    return dict(name=f"lognormal{shape[2]}x{shape[1]}x{shape[0]}", kappa=kappa, S=S, B=B, h=h,
                nside=nside, q=rotation_quaternion(seed) if rotate else IDENTITY_Q.copy(), Ib=None)


def cloud_problem(nx: int = 256, ny: int = 128, nz: int = 128, B: int = 16, nside: int = 8, seed: int = 3,
                  rotate: bool = True, kappa_amb: float = 1e-2, kappa_cloud: float = 1e3,
                  semi_axes=(0.1, 0.06, 0.06)):
    """Shadow-casting cloud; the beam on the x = 0 face depends on the
    direction set, so Ib is built by ``beam_ib`` once the directions exist."""
    h = 1.0 / ny
    Z, Y, X = _centres((nz, ny, nx), h)
    cx, cy, cz = 0.5 * nx * h, 0.5 * ny * h, 0.5 * nz * h
    ax, ay, az = semi_axes
    rho_e = np.sqrt(((X - cx) / ax) ** 2 + ((Y - cy) / ay) ** 2 + ((Z - cz) / az) ** 2)
    d = (rho_e - 1.0) * min(semi_axes)
    kappa = kappa_amb + (kappa_cloud - kappa_amb) * 0.5 * (1.0 - np.tanh(d / (2.0 * h)))
    S = np.zeros_like(kappa)
    return dict(name=f"cloud{nx}x{ny}x{nz}", kappa=kappa, S=S, B=B, h=h, nside=nside,
                q=rotation_quaternion(seed) if rotate else IDENTITY_Q.copy(), Ib=None,
                beam_half_angle_deg=10.0)


def beam_ib(dirs: np.ndarray, half_angle_deg: float = 10.0, face: int = 0, value: float = 1.0) -> np.ndarray:
    """Ib [6][ndir]: ``value`` on boundary face ``face`` (0 = x-low) for the
    directions within ``half_angle_deg`` of that face's inward normal, 0
    elsewhere."""
    normals = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], dtype=np.float64)
    cosang = dirs[:, :3] @ normals[face]
    Ib = np.zeros((6, dirs.shape[0]))
    Ib[face, cosang >= math.cos(math.radians(half_angle_deg))] = value
    return Ib


def batched_problems(n_grids: int = 64, seed0: int = 100, edges=(32, 48, 64, 80, 96), blocks=(8, 16),
                     nsides=(2, 4)):
    """Ragged batch: per grid an edge, block edge and nside drawn uniformly
    (seeded by the grid's own seed), each with its own lognormal fields."""
    out = []
    for g in range(n_grids):
        rng = np.random.default_rng(seed0 + g)
        n = int(rng.choice(edges))
        B = int(rng.choice(blocks))
        nside = int(rng.choice(nsides))
        out.append(lognormal_problem(n=n, B=B, nside=nside, seed=seed0 + g))
    return out


def _shift(g: np.ndarray, disp) -> np.ndarray:
    """g(x - disp) of a periodic field (disp in cells per axis, (x, y, z)),
    by a phase shift in Fourier space (exact for a band-limited field)."""
    nz, ny, nx = g.shape
    gk = np.fft.rfftn(g)
    kz = np.fft.fftfreq(nz)[:, None, None]
    ky = np.fft.fftfreq(ny)[None, :, None]
    kx = np.fft.rfftfreq(nx)[None, None, :]
    phase = np.exp(-2j * math.pi * (kx * disp[0] + ky * disp[1] + kz * disp[2]))
    return np.fft.irfftn(gk * phase, s=g.shape, axes=(0, 1, 2))


def lognormal_sequence(n: int = 128, B: int = 16, nside: int = 4, seed: int = 2, steps: int = 8,
                       cells_per_step: float = 0.05, direction=(1.0, 0.6, 0.3), **kw):
    """Time sequence of the lognormal workload for the reuse of f across time
    steps: the two Gaussian fields behind kappa and T are carried along
    ``direction`` by ``cells_per_step`` cells per step (periodic), the
    recipe of ``lognormal_problem`` applied to each shifted pair.  Returns
    the step-0 problem dict (its kappa, S are step 0's) and a list of
    (kappa, S) float32 arrays, one per step."""
    p = lognormal_problem(n=n, B=B, nside=nside, seed=seed, **kw)
    shape = p["kappa"].shape
    rng = np.random.default_rng(seed)
    g1 = gaussian_random_field(shape, rng)
    g2 = gaussian_random_field(shape, rng)
    sig_k = kw.get("sigma_ln_kappa", 1.5)
    sig_t = kw.get("sigma_ln_T", 0.5)
    rho = kw.get("rho", 0.5)
    med = kw.get("median_dtau", 10 ** -0.5)
    clip = kw.get("dtau_clip", (1e-3, 1e2))
    d = np.asarray(direction, float)
    d /= np.linalg.norm(d)
    seq = []
    for t in range(steps):
        disp = d * cells_per_step * t
        a1 = g1 if t == 0 else _shift(g1, disp)
        a2 = g2 if t == 0 else _shift(g2, disp)
        dtau = np.clip(np.exp(math.log(med) + sig_k * a1), clip[0], clip[1])
        lnT = sig_t * (rho * a1 + math.sqrt(1.0 - rho * rho) * a2)
        seq.append((np.ascontiguousarray((dtau / p["h"]).astype(np.float32)),
                    np.ascontiguousarray((np.exp(4.0 * lnT) / FOUR_PI).astype(np.float32))))
    return p, seq
