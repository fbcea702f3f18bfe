"""Pins of the local-closure oracle (oracle/local_closures.py; paper Sec. 4.1):
limits of the Eddington factor, the tensor's trace and eigenstructure, free
streaming, isotropy, rotation covariance and the clipping reading.  A wrong
coefficient, sign or component order breaks one of them."""
import math

import numpy as np

from oracle import local_closures as lc


def _tensor(T, c):
    xx, yy, zz, xy, xz, yz = T[:, c]
    return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]])


def _moments(E, F):
    M = np.zeros((10, len(E)))
    M[0] = E
    M[1:4] = np.asarray(F).T
    return M


def test_eddington_factor_limits_and_shape():
    assert lc.chi(0.0) == 1.0 / 3.0           # isotropic: 3 / 9
    assert abs(lc.chi(1.0) - 1.0) < 1e-15      # free streaming: 7 / 7
    fs = np.linspace(0.0, 1.0, 101)
    x = np.array([lc.chi(f) for f in fs])
    assert np.all(np.diff(x) > 0)              # rises monotonically from 1/3 to 1
    # even in f: flat at f = 0
    assert abs(lc.chi(1e-4) - 1.0 / 3.0) < 1e-8


def test_trace_one_and_flux_direction_is_an_eigenvector():
    rng = np.random.default_rng(1)
    n = 200
    E = rng.uniform(0.1, 2.0, n)
    F = rng.normal(size=(n, 3))
    F *= (rng.uniform(0.0, 1.0, n) * E / np.linalg.norm(F, axis=1))[:, None]
    T = lc.m1(_moments(E, F))
    for c in range(n):
        t = _tensor(T, c)
        assert abs(np.trace(t) - 1.0) < 1e-14
        f = np.linalg.norm(F[c]) / E[c]
        nhat = F[c] / np.linalg.norm(F[c])
        x = lc.chi(f)
        np.testing.assert_allclose(t @ nhat, x * nhat, atol=1e-14)  # eigenvalue chi along n
        w = np.linalg.eigvalsh(t)
        np.testing.assert_allclose(sorted(w), sorted([x, (1 - x) / 2, (1 - x) / 2]), atol=1e-14)


def test_free_streaming_gives_n_outer_n_and_isotropy_gives_a_third():
    n = np.array([1.0, -2.0, 2.0]) / 3.0
    T = lc.m1(_moments([2.0, 1.0, 0.0, 3.0], [2.0 * n, [0, 0, 0], [0.5, 0, 0], 5.0 * n]))
    np.testing.assert_allclose(_tensor(T, 0), np.outer(n, n), atol=1e-15)
    np.testing.assert_allclose(_tensor(T, 1), np.eye(3) / 3, atol=1e-15)   # F = 0
    np.testing.assert_allclose(_tensor(T, 2), np.eye(3) / 3, atol=1e-15)   # E = 0
    np.testing.assert_allclose(_tensor(T, 3), np.outer(n, n), atol=1e-15)  # |F| > E: clipped to f = 1
    np.testing.assert_allclose(lc.eddington(4)[:, 0], [1 / 3, 1 / 3, 1 / 3, 0, 0, 0])


def test_rotation_covariance():
    rng = np.random.default_rng(2)
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    F = np.array([[0.3, -0.2, 0.5]])
    T0 = _tensor(lc.m1(_moments([1.0], F)), 0)
    T1 = _tensor(lc.m1(_moments([1.0], F @ R.T)), 0)
    np.testing.assert_allclose(T1, R @ T0 @ R.T, atol=1e-14)


def test_half_flux_by_hand():
    # f = 1/2: chi = (3 + 1) / (5 + 2 sqrt(13/4)) = 4 / (5 + sqrt 13)
    x = 4.0 / (5.0 + math.sqrt(13.0))
    T = lc.m1(_moments([2.0], [[0.0, 0.0, 1.0]]))
    np.testing.assert_allclose(T[:, 0], [(1 - x) / 2, (1 - x) / 2, x, 0, 0, 0], atol=1e-15)
