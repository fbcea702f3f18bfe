"""Pins for the oracle's direction set (VETTAM Sec. 2.2.5 and App. B: HEALPix
directions, N = 12 nside^2, equal weights, random rotation)."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _ring_table(nside):
    """(z, pixel count) for every HEALPix ring, exact rationals, from the
    ring-scheme closed forms (Gorski et al. 2005, Sec. 4)."""
    rings = []
    for i in range(1, 4 * nside):
        if i < nside:
            rings.append((1 - Fraction(i * i, 3 * nside * nside), 4 * i))
        elif i <= 3 * nside:
            rings.append((Fraction(4, 3) - Fraction(2 * i, 3 * nside), 4 * nside))
        else:
            ii = 4 * nside - i
            rings.append((-(1 - Fraction(ii * ii, 3 * nside * nside)), 4 * ii))
    return rings


@pytest.mark.parametrize("nside", [1, 2, 4, 8])
def test_counts_weights_and_balance(ora, nside):
    d = ora.healpix(nside)
    N = 12 * nside * nside
    assert d.shape == (N, 4)
    np.testing.assert_allclose(d[:, 3], 4 * math.pi / N, rtol=0, atol=1e-15)
    assert abs(d[:, 3].sum() - 4 * math.pi) < 1e-12
    np.testing.assert_allclose(np.linalg.norm(d[:, :3], axis=1), 1.0, atol=1e-15)
    # sum_k w_k n_k = 0: HEALPix is symmetric under n -> -n
    assert np.abs((d[:, 3:] * d[:, :3]).sum(0)).max() < 1e-14


@pytest.mark.parametrize("nside", [1, 2, 4, 8])
def test_ring_z_values_match_closed_form(ora, nside):
    d = ora.healpix(nside)
    got = np.sort(d[:, 2])[::-1]
    want = []
    for z, cnt in _ring_table(nside):
        want += [float(z)] * cnt
    np.testing.assert_allclose(got, np.array(want), atol=1e-15)


@pytest.mark.parametrize("nside", [1, 2, 4, 8])
def test_quadrature_tensor_closed_form(ora, nside):
    """Q = sum w n n / sum w: diagonal with Qzz = <z^2> over the rings (exact
    rational) and Qxx = Qyy = (1 - Qzz)/2; off-diagonals vanish."""
    d = ora.healpix(nside)
    Q = np.einsum("k,ki,kj->ij", d[:, 3], d[:, :3], d[:, :3]) / d[:, 3].sum()
    N = 12 * nside * nside
    qzz = sum(cnt * z * z for z, cnt in _ring_table(nside)) / N
    want = np.diag([float((1 - qzz) / 2), float((1 - qzz) / 2), float(qzz)])
    np.testing.assert_allclose(Q, want, atol=1e-15)
    if nside == 1:
        assert abs(Q[2, 2] - 8 / 27) < 1e-15 and abs(Q[0, 0] - 19 / 54) < 1e-15


def test_nside1_matches_hand_worked_table(ora):
    want = np.loadtxt(os.path.join(GOLDEN, "healpix_nside1.txt"))
    got = ora.healpix(1)[:, :3]
    np.testing.assert_allclose(got, want, atol=1e-14)


def test_rotation_is_the_quaternion_rotation(ora):
    from scipy.spatial.transform import Rotation

    from paper_2202_08778_gb300 import synth

    q = synth.rotation_quaternion(7)
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()  # scipy: (x, y, z, w)
    base = ora.healpix(4)
    rot = ora.healpix(4, q)
    np.testing.assert_allclose(rot[:, :3], base[:, :3] @ R.T, atol=1e-14)
    np.testing.assert_allclose(rot[:, 3], base[:, 3])
    # identity quaternion leaves the set unchanged
    np.testing.assert_allclose(ora.healpix(4, [1, 0, 0, 0]), base, atol=0)


def test_bad_nside_rejected(ora):
    for bad in (0, 3, 6, -2):
        with pytest.raises(ValueError):
            ora.healpix(bad)
