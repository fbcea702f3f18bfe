"""Pins for the oracle's angular quadratures (VETTAM Eqs. 10-12 and the
discrete sums of Sec. 2.2.5, Eqs. 55-56, c = 1) and closure f = P/E (Eq. 13)."""
import math

import numpy as np

from paper_2202_08778_gb300 import synth


def test_single_direction_moments(ora):
    """I_k = delta_{k k0}: E = w, F = w n, P = w n n, component by
    component in the stated order (E, Fx, Fy, Fz, Pxx, Pyy, Pzz, Pxy, Pxz, Pyz)."""
    dirs = ora.healpix(2, synth.rotation_quaternion(3))
    for k0 in (0, 13, 47):
        I = np.zeros((48, 2, 3))
        I[k0] = 2.0
        M = ora.moments(I, dirs)
        w = dirs[k0, 3]
        x, y, z = dirs[k0, :3]
        want = [1, x, y, z, x * x, y * y, z * z, x * y, x * z, y * z]
        for m in range(10):
            np.testing.assert_allclose(M[m], 2.0 * w * want[m], rtol=1e-15, atol=1e-17)


def test_isotropic_field_moments(ora):
    """I_k = c: E = 4 pi c, F = 0, and f = Q (the quadrature tensor, whose
    unrotated closed form is pinned in test_oracle_directions)."""
    dirs = ora.healpix(4)
    I = np.full((192, 3, 1), 1.75)
    M = ora.moments(I, dirs)
    np.testing.assert_allclose(M[0], 4 * math.pi * 1.75, rtol=1e-14)
    assert np.abs(M[1:4]).max() < 1e-13
    f, iso = ora.closure(M)
    Q = np.einsum("k,ki,kj->ij", dirs[:, 3], dirs[:, :3], dirs[:, :3]) / (4 * math.pi)
    np.testing.assert_allclose(f[0], Q[0, 0], atol=1e-14)
    np.testing.assert_allclose(f[2], Q[2, 2], atol=1e-14)
    assert np.abs(f[3:]).max() < 1e-14
    assert not iso.any()


def test_closure_invariants_random_positive_intensities(ora):
    rng = np.random.default_rng(5)
    dirs = ora.healpix(4, synth.rotation_quaternion(5))
    I = rng.lognormal(0.0, 2.0, (192, 50))
    M = ora.moments(I, dirs)
    f, iso = ora.closure(M)
    np.testing.assert_allclose(f[0] + f[1] + f[2], 1.0, atol=1e-14)
    # |F| <= E (c = 1)
    assert (np.sqrt((M[1:4] ** 2).sum(0)) <= M[0] * (1 + 1e-14)).all()
    # eigenvalues of f in [0, 1]
    for c in range(50):
        T = np.array([[f[0, c], f[3, c], f[4, c]], [f[3, c], f[1, c], f[5, c]], [f[4, c], f[5, c], f[2, c]]])
        ev = np.linalg.eigvalsh(T)
        assert ev.min() >= -1e-14 and ev.max() <= 1 + 1e-14


def test_closure_floor_gives_isotropic_tensor(ora):
    """Where no radiation arrives (E = 0) or E is below 1e-30 of the maximum,
    f falls back to I/3 and the cell is flagged."""
    dirs = ora.healpix(1)
    I = np.zeros((12, 3))
    I[:, 0] = 1.0
    I[3, 2] = 1e-40
    M = ora.moments(I, dirs)
    f, iso = ora.closure(M, floor_rel=1e-30)
    assert list(iso) == [0, 1, 1]
    np.testing.assert_allclose(f[:3, 1:], 1.0 / 3.0)
    np.testing.assert_allclose(f[3:, 1:], 0.0)
