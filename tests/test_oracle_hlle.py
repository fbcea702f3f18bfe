"""Pins of the HLLE wavespeed oracle (oracle/hlle.py; paper Sec. 2.2.3 and
App. A): the free-streaming and thick limits, a value worked by hand, the
interface average, symmetry, boundary faces and the degenerate tensors.  A
dropped factor 10 or 2, a swapped f and kappa, a wrong face indexing or the
minimum instead of the maximum free-streaming factor breaks one of them."""
import math

import numpy as np

from oracle import hlle


def test_free_streaming_limit_is_the_eigenvalue():
    # kappa = 0: tau = 0, the correction is 1, the speed sqrt(f) c
    for f, c in ((1.0, 1.0), (1.0 / 3.0, 2.0), (0.81, 3e10)):
        assert hlle.face_speed(f, 0.0, f, 0.0, 0.25, c) == math.sqrt(f) * c


def test_thick_limit_follows_one_over_root_tau():
    # tau >> 1: g -> 1/sqrt(tau), so C -> sqrt(f) c sqrt(2 f) / (10 h kappa)
    f, h, c = 1.0 / 3.0, 0.01, 1.0
    for kappa in (1e3, 1e4, 1e5):
        want = math.sqrt(f) * c * math.sqrt(2.0 * f) / (10.0 * h * kappa)
        got = hlle.face_speed(f, kappa, f, kappa, h, c)
        tau = (10 * h * kappa) ** 2 / (2 * f)
        assert abs(got / want - 1.0) <= math.exp(-tau) + 1e-15


def test_value_worked_by_hand():
    # f = 1/3, h kappa = 0.1: tau = (10 * 0.1)^2 / (2/3) = 1.5,
    # g = sqrt((1 - e^-1.5) / 1.5) = sqrt(0.7768698398515702 / 1.5),
    # C = sqrt(1/3) g
    g = math.sqrt(0.7768698398515702 / 1.5)
    assert abs(hlle.face_speed(1 / 3, 10.0, 1 / 3, 10.0, 0.01) - g / math.sqrt(3.0)) < 1e-15
    assert abs(g / math.sqrt(3.0) - 0.4154970) < 1e-7


def test_interface_average_and_symmetry():
    fL, kL, fR, kR, h = 0.5, 3.0, 0.2, 40.0, 0.02
    tauL = (10 * h * kL) ** 2 / (2 * fL)
    tauR = (10 * h * kR) ** 2 / (2 * fR)
    tau = 0.5 * (tauL + tauR)
    want = math.sqrt(0.5) * math.sqrt(-math.expm1(-tau) / tau)  # the larger sqrt(f)
    assert abs(hlle.face_speed(fL, kL, fR, kR, h) - want) < 1e-15
    assert hlle.face_speed(fL, kL, fR, kR, h) == hlle.face_speed(fR, kR, fL, kL, h)


def test_degenerate_tensors():
    assert hlle.face_speed(0.0, 5.0, 0.0, 5.0, 0.1) == 0.0       # no radiation along the axis
    assert hlle.face_speed(0.0, 0.0, 0.0, 0.0, 0.1) == 0.0
    # one side with f_aa = 0: tau = inf on that side, the interface mean is inf
    assert hlle.face_speed(0.0, 1.0, 0.6, 1.0, 0.1) == 0.0
    # kappa = 0 on one side only: the mean is half the other side's tau
    t = (10 * 0.1 * 2.0) ** 2 / (2 * 0.5)
    assert abs(hlle.face_speed(0.5, 0.0, 0.5, 2.0, 0.1) - math.sqrt(0.5) * math.sqrt(-math.expm1(-t / 2) / (t / 2))) < 1e-15


def test_grid_faces_per_axis_and_boundaries():
    rng = np.random.default_rng(4)
    nz, ny, nx, h = 3, 4, 5, 0.1
    f = np.zeros((6, nz, ny, nx))
    f[:3] = rng.uniform(0.05, 0.9, (3, nz, ny, nx))
    k = rng.lognormal(0.0, 1.0, (nz, ny, nx))
    for axis in range(3):
        C = hlle.wavespeeds(f, k, h, axis)
        shape = [nz, ny, nx]
        shape[2 - axis] += 1
        assert C.shape == tuple(shape)
        faa = f[axis]
        # an interior face and both boundary faces, indexed by hand
        if axis == 0:
            assert C[1, 2, 3] == hlle.face_speed(faa[1, 2, 2], k[1, 2, 2], faa[1, 2, 3], k[1, 2, 3], h)
            assert C[1, 2, 0] == hlle.face_speed(faa[1, 2, 0], k[1, 2, 0], faa[1, 2, 0], k[1, 2, 0], h)
            assert C[1, 2, nx] == hlle.face_speed(faa[1, 2, nx - 1], k[1, 2, nx - 1], faa[1, 2, nx - 1], k[1, 2, nx - 1], h)
        elif axis == 1:
            assert C[2, 1, 4] == hlle.face_speed(faa[2, 0, 4], k[2, 0, 4], faa[2, 1, 4], k[2, 1, 4], h)
            assert C[2, ny, 4] == hlle.face_speed(faa[2, ny - 1, 4], k[2, ny - 1, 4], faa[2, ny - 1, 4], k[2, ny - 1, 4], h)
        else:
            assert C[1, 3, 0] == hlle.face_speed(faa[0, 3, 0], k[0, 3, 0], faa[1, 3, 0], k[1, 3, 0], h)
            assert C[0, 3, 0] == hlle.face_speed(faa[0, 3, 0], k[0, 3, 0], faa[0, 3, 0], k[0, 3, 0], h)


def test_uniform_isotropic_state_gives_one_speed():
    f = np.zeros((6, 2, 2, 3))
    f[:3] = 1.0 / 3.0
    k = np.full((2, 2, 3), 7.0)
    want = hlle.face_speed(1 / 3, 7.0, 1 / 3, 7.0, 0.05)
    for axis in range(3):
        assert np.all(hlle.wavespeeds(f, k, 0.05, axis) == want)
