"""Pins of the change-gate oracle (oracle/field_change.py; the reuse of f
across time steps of paper Sec. 4.2): the opacity measure against the exact
change of a cell's transmission (an upper bound everywhere, equal to the
optical-depth change for thin cells, negligible for thick ones), block
numbering and maxima against brute-force loops over cells, exact values of
single-cell perturbations of either sign, symmetry, non-finite inputs, scale
invariance of the decision, and the decision table."""
import math

import numpy as np
import pytest

from oracle import field_change as fc


def _brute(kappa, S, kr, sr, h, B):
    """Per-cell loop with the block index from integer division."""
    nz, ny, nx = kappa.shape
    nbx, nby = nx // B, ny // B
    nb = nbx * nby * (nz // B)
    out = np.zeros((nb, 3))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                b = i // B + nbx * (j // B + nby * (k // B))
                a = np.float32(kappa[k, j, i]) * np.float32(h)
                c = np.float32(kr[k, j, i]) * np.float32(h)
                dt = abs(a - c) / ((1 + a / 2) * (1 + c / 2))
                ds = float(abs(np.float32(S[k, j, i]) - np.float32(sr[k, j, i])))
                out[b, 0] = max(out[b, 0], np.float32(dt))
                out[b, 1] = max(out[b, 1], ds)
                out[b, 2] = max(out[b, 2], abs(float(sr[k, j, i])))
    return out


def _fields(shape, seed):
    rng = np.random.default_rng(seed)
    k = rng.lognormal(0.0, 1.0, shape).astype(np.float32)
    s = rng.lognormal(0.0, 1.0, shape).astype(np.float32)
    kr = (k * rng.uniform(0.9, 1.1, shape)).astype(np.float32)
    sr = (s * rng.uniform(0.9, 1.1, shape)).astype(np.float32)
    return k, s, kr, sr


def _per_cell(a, b, h):
    """The opacity measure of optical depths a -> b, one 2^3 block each."""
    n = a.size
    k = np.repeat(np.float32(a / h), 2).reshape(1, 1, 2 * n).repeat(2, 0).repeat(2, 1)
    kr = np.repeat(np.float32(b / h), 2).reshape(1, 1, 2 * n).repeat(2, 0).repeat(2, 1)
    one = np.ones_like(k)
    return fc.change(k, one, kr, one, h, 2)[3::3], np.float64(k[0, 0, ::2] * np.float32(h)), \
        np.float64(kr[0, 0, ::2] * np.float32(h))


def test_opacity_measure_bounds_the_change_of_transmission():
    rng = np.random.default_rng(7)
    a = np.exp(rng.uniform(-12, 5, 4096))                # optical depths 6e-6 .. 150
    b = a * np.exp(rng.normal(0, 0.5, 4096))
    got, aa, bb = _per_cell(a, b, 0.5)
    exact = np.abs(np.exp(-aa) - np.exp(-bb))
    assert np.all(got >= exact * (1 - 1e-5))               # an upper bound
    thin = np.maximum(aa, bb) < 1e-3
    assert thin.sum() > 100
    np.testing.assert_allclose(got[thin], np.abs(aa - bb)[thin], rtol=2e-3)   # ~ |dtau| when thin
    # thick cells: a large change of optical depth barely counts (50 -> 60: 10 / (26 * 31))
    got, aa, bb = _per_cell(np.array([50.0]), np.array([60.0]), 0.5)
    assert got[0] == np.float32(10.0) / np.float32(26.0 * 31.0)


@pytest.mark.parametrize("shape,B", [((4, 6, 8), 2), ((6, 3, 9), 3), ((8, 8, 4), 4)])
def test_blocks_match_a_loop_over_cells(shape, B):
    k, s, kr, sr = _fields(shape, 1)
    h = 0.37
    got = fc.change(k, s, kr, sr, h, B)
    ref = _brute(k, s, kr, sr, h, B)
    np.testing.assert_array_equal(got[3:].reshape(-1, 3), ref.astype(np.float32))
    np.testing.assert_array_equal(got[:3], ref.max(axis=0).astype(np.float32))


@pytest.mark.parametrize("delta", [0.5, -0.5])
def test_single_cell_perturbation_lands_in_its_block_only(delta):
    shape, B, h = (6, 4, 8), 2, 0.25
    k = np.ones(shape, np.float32)
    s = np.full(shape, 3.0, np.float32)
    kp, sp = k.copy(), s.copy()
    kp[5, 2, 7] += delta       # block (i 3, j 1, k 2) -> 3 + 4 * (1 + 2 * 2) = 23
    # a = (1 + delta) / 4, b = 1/4: |a - b| / ((1 + a/2)(1 + b/2)) =
    # (1/8) / ((19/16)(9/8)) = 16/171 for delta = 1/2, (1/8) / ((17/16)(9/8)) = 16/153 for -1/2
    dtrans = np.float32(16 / 171) if delta > 0 else np.float32(16 / 153)
    sp[0, 3, 0] -= 2 * delta   # block (0, 1, 0) -> 4
    got = fc.change(kp, sp, k, s, h, B)
    per = got[3:].reshape(-1, 3)
    assert per.shape[0] == 4 * 2 * 3
    want_tau = np.zeros(per.shape[0], np.float32)
    want_tau[23] = dtrans
    want_s = np.zeros(per.shape[0], np.float32)
    want_s[4] = 1.0
    np.testing.assert_array_equal(per[:, 0], want_tau)
    np.testing.assert_array_equal(per[:, 1], want_s)
    np.testing.assert_array_equal(per[:, 2], np.float32(3.0))
    np.testing.assert_array_equal(got[:3], np.array([dtrans, 1.0, 3.0], np.float32))


def test_unchanged_fields_give_zero_change_and_the_source_scale():
    k, s, _, _ = _fields((4, 4, 4), 2)
    s[1, 2, 3] = -7.5
    got = fc.change(k, s, k, s, 1.0, 2)
    assert np.all(got[3:].reshape(-1, 3)[:, :2] == 0.0)
    assert got[2] == np.float32(max(7.5, np.abs(s).max()))


def test_change_is_symmetric_in_current_and_reference():
    k, s, kr, sr = _fields((4, 6, 4), 3)
    a = fc.change(k, s, kr, sr, 0.1, 2).reshape(-1, 3)
    b = fc.change(kr, sr, k, s, 0.1, 2).reshape(-1, 3)
    np.testing.assert_array_equal(a[:, :2], b[:, :2])


def test_non_finite_inputs_count_as_infinite_change():
    k, s, kr, sr = _fields((4, 4, 4), 4)
    k[0, 0, 0] = np.nan
    s[3, 3, 3] = np.inf
    sr[3, 3, 3] = np.inf          # inf - inf = nan -> inf
    got = fc.change(k, s, kr, sr, 0.5, 2)
    per = got[3:].reshape(-1, 3)
    assert per[0, 0] == np.inf and per[7, 1] == np.inf and per[7, 2] == np.inf
    assert np.all(np.isfinite(per[1:7]))
    assert fc.recompute(got[:3], age=1, first=False, tol_tau=1e9, tol_S=1e9, max_age=100)


def test_decision_is_invariant_under_scaling_the_source():
    k, s, kr, sr = _fields((4, 4, 4), 5)
    a = fc.change(k, s, kr, sr, 0.2, 2)
    b = fc.change(k, 4 * s, kr, 4 * sr, 0.2, 2)
    np.testing.assert_array_equal(b[1::3], 4 * a[1::3])   # dS
    np.testing.assert_array_equal(b[2::3], 4 * a[2::3])   # Sref
    for tol in (1e-3, 0.05, 0.2):
        assert fc.recompute(a[:3], 1, False, 1e9, tol, 100) == fc.recompute(b[:3], 1, False, 1e9, tol, 100)


@pytest.mark.parametrize("triple,age,first,expect", [
    ((0.0, 0.0, 1.0), 0, True, True),           # nothing stored yet
    ((0.0, 0.0, 1.0), 3, False, False),          # unchanged, young
    ((0.0, 0.0, 1.0), 4, False, True),           # max_age reached
    ((0.011, 0.0, 1.0), 1, False, True),         # optical depth moved
    ((0.01, 0.0, 1.0), 1, False, False),         # exactly at the tolerance: reuse
    ((0.0, 0.0201, 2.0), 1, False, True),        # source moved by more than 1% of its scale
    ((0.0, 0.02, 2.0), 1, False, False),
    ((math.inf, 0.0, 1.0), 1, False, True),
])
def test_decision_table(triple, age, first, expect):
    assert fc.recompute(np.float32(triple), age, first, tol_tau=0.01, tol_S=0.01, max_age=4) is expect


def test_block_edge_must_divide_the_grid():
    k = np.ones((4, 4, 6), np.float32)
    with pytest.raises(ValueError):
        fc.change(k, k, k, k, 1.0, 4)
