"""Pins for the oracle's formal solution of the gray transfer equation
dI/ds = kappa (S - I) (VETTAM Eq. 14) by hybrid characteristics, and for its
moments and closure (Eqs. 10-13).  Every expected value below comes from a
closed form, an invariant of the equation, or the brute-force integrator in
tests/bruteforce.py -- never from the oracle itself."""
import math

import numpy as np
import pytest

from bruteforce import bf_trace
from paper_2202_08778_gb300 import synth


def _rng(seed):
    return np.random.default_rng(seed)


def _dirs(ora, nside, seed=None):
    return ora.healpix(nside, None if seed is None else synth.rotation_quaternion(seed))


def _upwind_distance(shape, dirs):
    """[ndir][nz][ny][nx] distance (cell units) from each cell centre back to
    the domain boundary along -n, and the axis of the face it reaches."""
    nz, ny, nx = shape
    Z, Y, X = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    P = [X, Y, Z]
    dims = [nx, ny, nz]
    out, axis = [], []
    for n in dirs[:, :3]:
        ts = []
        for a in range(3):
            if n[a] > 0:
                ts.append(P[a] / n[a])
            elif n[a] < 0:
                ts.append((dims[a] - P[a]) / -n[a])
            else:
                ts.append(np.full(X.shape, np.inf))
        ts = np.stack(ts)
        out.append(ts.min(0))
        axis.append(ts.argmin(0))
    return np.array(out), np.array(axis)


def test_constant_state_is_preserved_multiblock(ora):
    """I = S everywhere is the solution when S and the inflow equal one
    constant, whatever kappa is; interpolation must not disturb it."""
    rng = _rng(11)
    shape = (8, 12, 16)
    kappa = rng.uniform(0.0, 30.0, shape)
    S = np.full(shape, 2.5)
    dirs = _dirs(ora, 2, seed=5)
    Ib = np.full((6, dirs.shape[0]), 2.5)
    I = ora.trace(kappa, S, dirs, B=4, h=1 / 16, Ib=Ib)
    np.testing.assert_allclose(I, 2.5, rtol=0, atol=1e-13)


def test_beam_in_vacuum_gives_n_outer_n(ora):
    """kappa = 0 and one direction k0 lit from every face: I_k0 = 1, all
    other I_k = 0, so E = w_k0 and f = n_k0 n_k0 exactly."""
    shape = (8, 8, 8)
    dirs = _dirs(ora, 2, seed=9)
    for k0 in (0, 17, 40):
        Ib = np.zeros((6, dirs.shape[0]))
        Ib[:, k0] = 1.0
        f, M, I, iso = ora.vet_closure(np.zeros(shape), np.zeros(shape), dirs, B=4, h=0.1, Ib=Ib)
        np.testing.assert_allclose(I[k0], 1.0, rtol=0, atol=1e-15)  # bilinear weights sum to 1
        assert np.abs(np.delete(I, k0, axis=0)).max() == 0.0
        n = dirs[k0, :3]
        want = [n[0] * n[0], n[1] * n[1], n[2] * n[2], n[0] * n[1], n[0] * n[2], n[1] * n[2]]
        for m in range(6):
            np.testing.assert_allclose(f[m], want[m], atol=2e-15)
        np.testing.assert_allclose(M[0], dirs[k0, 3], rtol=1e-15 * 4)
        assert not iso.any()


@pytest.mark.parametrize("nside,seed", [(1, None), (2, 3), (4, 4)])
def test_single_block_uniform_medium_closed_form(ora, nside, seed):
    """One block covering the grid is pure long characteristics: with uniform
    kappa, S and vacuum inflow, I = S (1 - exp(-kappa h d)) where d is the
    distance from the cell centre back to the domain boundary."""
    kappa, S0, h = 1.7, 0.8, 0.3
    shape = (6, 6, 6)  # one cubic block of edge 6
    dirs = _dirs(ora, nside, seed)
    I = ora.trace(np.full(shape, kappa), np.full(shape, S0), dirs, B=6, h=h)
    d, _ = _upwind_distance(shape, dirs)
    want = S0 * (1.0 - np.exp(-kappa * h * d))
    np.testing.assert_allclose(I, want, rtol=1e-13, atol=1e-15)


def test_single_block_pure_absorber_closed_form(ora):
    """S = 0, I = 1 entering through x = 0 only: I = exp(-kappa h x/n_x) for
    cells whose backward ray reaches x = 0 first, else 0."""
    shape = (8, 8, 8)
    kappa, h = 2.3, 0.05
    dirs = _dirs(ora, 4, seed=21)
    Ib = np.zeros((6, dirs.shape[0]))
    Ib[0, :] = 1.0
    I = ora.trace(np.full(shape, kappa), np.zeros(shape), dirs, B=8, h=h, Ib=Ib)
    d, ax = _upwind_distance(shape, dirs)
    lit = (ax == 0) & (dirs[:, 0] > 0)[:, None, None, None]
    want = np.where(lit, np.exp(-kappa * h * d), 0.0)
    np.testing.assert_allclose(I, want, rtol=1e-13, atol=1e-300)


def test_single_block_emitting_slab_closed_form(ora):
    """kappa, S nonzero only in the cell slab a <= x < b, vacuum elsewhere:
    behind the slab, a ray that crosses it completely inside the domain
    carries I = S (1 - exp(-kappa h (b - a)/n_x))."""
    n, a, b = 12, 3, 6
    shape = (n, n, n)
    kap, S0, h = 0.9, 1.3, 0.2
    kappa = np.zeros(shape)
    S = np.zeros(shape)
    kappa[:, :, a:b] = kap
    S[:, :, a:b] = S0
    dirs = _dirs(ora, 4, seed=8)
    I = ora.trace(kappa, S, dirs, B=n, h=h)
    nz, ny, nx = shape
    Z, Y, X = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    checked = 0
    for k, nvec in enumerate(dirs[:, :3]):
        if nvec[0] <= 0.05:
            continue
        t_a = (X - a) / nvec[0]  # reach x = a going backward
        ok = X > b
        for ax_, P, dim in ((1, Y, ny), (2, Z, nz)):
            if nvec[ax_] > 0:
                ok &= P - t_a * nvec[ax_] >= 0
            elif nvec[ax_] < 0:
                ok &= P - t_a * nvec[ax_] <= dim
        want = S0 * (1 - math.exp(-kap * h * (b - a) / nvec[0]))
        np.testing.assert_allclose(I[k][ok], want, rtol=1e-13)
        checked += int(ok.sum())
    assert checked > 1000


@pytest.mark.parametrize("shape,B,nside,seed", [((4, 4, 6), 2, 1, 31), ((4, 4, 4), 4, 1, 32), ((6, 3, 3), 3, 1, 33)])
def test_hybrid_matches_bruteforce(ora, shape, B, nside, seed):
    """Multi-block hybrid characteristics vs an independent fine-step
    restatement of the same reading (different geometry code path)."""
    rng = _rng(seed)
    h = 0.25
    kappa = rng.uniform(1.0, 4.0, shape)
    S = rng.uniform(0.5, 2.0, shape)
    dirs = _dirs(ora, nside, seed)
    Ib = rng.uniform(0.0, 1.0, (6, dirs.shape[0]))
    I = ora.trace(kappa, S, dirs, B=B, h=h, Ib=Ib)
    ref = bf_trace(kappa, S, dirs, B, h, Ib, step=5e-4)
    np.testing.assert_allclose(I, ref, rtol=2e-3, atol=1e-6)


def test_bruteforce_check_is_sensitive(ora):
    """The brute-force comparison above fails for a planted mistake: an oracle
    that confused the y and z axes (emulated by exchanging the y and z
    components of every direction and the matching boundary faces) misses the
    brute-force answer by far more than the comparison's tolerance."""
    rng = _rng(41)
    shape, B, h = (4, 4, 6), 2, 0.25
    kappa = rng.uniform(1.0, 4.0, shape)
    S = rng.uniform(0.5, 2.0, shape)
    dirs = _dirs(ora, 1, 41)
    Ib = rng.uniform(0.0, 1.0, (6, dirs.shape[0]))
    ref = bf_trace(kappa, S, dirs, B, h, Ib, step=5e-4)
    # a wrong answer: trace with the y and z components of n exchanged
    bad_dirs = dirs.copy()
    bad_dirs[:, [1, 2]] = dirs[:, [2, 1]]
    Ib_bad = Ib.copy()
    Ib_bad[[2, 3, 4, 5]] = Ib[[4, 5, 2, 3]]
    bad = ora.trace(kappa, S, bad_dirs, B=B, h=h, Ib=Ib_bad)
    assert np.abs(bad - ref).max() / np.abs(ref).max() > 1e-2


def test_linearity_in_sources_and_inflow(ora):
    rng = _rng(51)
    shape = (8, 8, 8)
    kappa = rng.uniform(0.1, 10.0, shape)
    dirs = _dirs(ora, 2, 51)
    S1, S2 = rng.uniform(0, 1, shape), rng.uniform(0, 3, shape)
    Ib1, Ib2 = rng.uniform(0, 1, (6, 48)), rng.uniform(0, 2, (6, 48))
    a, b = 0.7, -1.9
    I1 = ora.trace(kappa, S1, dirs, 4, 0.125, Ib1)
    I2 = ora.trace(kappa, S2, dirs, 4, 0.125, Ib2)
    I12 = ora.trace(kappa, a * S1 + b * S2, dirs, 4, 0.125, a * Ib1 + b * Ib2)
    np.testing.assert_allclose(I12, a * I1 + b * I2, rtol=1e-12, atol=1e-12)


def test_mirror_symmetry(ora):
    """Reflecting the grid in x and the directions' x components permutes the
    solution exactly (inflow faces x-low and x-high swap)."""
    rng = _rng(61)
    shape = (8, 8, 12)
    kappa = rng.uniform(0.1, 10.0, shape)
    S = rng.uniform(0.0, 2.0, shape)
    dirs = _dirs(ora, 2, 61)
    Ib = rng.uniform(0, 1, (6, dirs.shape[0]))
    I = ora.trace(kappa, S, dirs, 4, 0.1, Ib)
    md = dirs.copy()
    md[:, 0] = -md[:, 0]
    mIb = Ib[[1, 0, 2, 3, 4, 5]]
    Im = ora.trace(kappa[:, :, ::-1], S[:, :, ::-1], md, 4, 0.1, mIb)
    np.testing.assert_allclose(Im[:, :, :, ::-1], I, rtol=1e-12, atol=1e-14)


def test_maximum_principle(ora):
    rng = _rng(71)
    shape = (8, 8, 8)
    kappa = rng.uniform(0.0, 20.0, shape)
    S = rng.uniform(0.3, 2.0, shape)
    dirs = _dirs(ora, 2, 71)
    Ib = rng.uniform(0.1, 1.5, (6, 48))
    I = ora.trace(kappa, S, dirs, 4, 0.1, Ib)
    lo, hi = min(S.min(), Ib.min()), max(S.max(), Ib.max())
    assert I.min() >= lo - 1e-14 and I.max() <= hi + 1e-14


def test_hybrid_approaches_long_characteristics_as_blocks_grow(ora):
    """Block edge B -> N turns hybrid into long characteristics; the gap must
    shrink monotonically on a smooth problem."""
    p = synth.blob_problem(n=16, B=16, nside=2, seed=1)
    dirs = _dirs(ora, 2, 1)
    ref = ora.trace(p["kappa"], p["S"], dirs, 16, p["h"])
    errs = []
    for B in (2, 4, 8):
        I = ora.trace(p["kappa"], p["S"], dirs, B, p["h"])
        errs.append(np.abs(I - ref).max() / np.abs(ref).max())
    assert errs[0] > errs[1] > errs[2] > 0


def test_thread_count_does_not_change_results(ora):
    p = synth.blob_problem(n=16, B=8, nside=2, seed=1)
    dirs = _dirs(ora, 2, 1)
    a = ora.trace(p["kappa"], p["S"], dirs, 8, p["h"], nthreads=1)
    b = ora.trace(p["kappa"], p["S"], dirs, 8, p["h"], nthreads=5)
    np.testing.assert_array_equal(a, b)


def test_invalid_grids_rejected(ora):
    dirs = _dirs(ora, 1)
    with pytest.raises(ValueError):
        ora.trace(np.ones((6, 6, 6)), np.ones((6, 6, 6)), dirs, B=4, h=0.1)
    with pytest.raises(ValueError):
        ora.trace(np.ones((4, 4, 4)), np.ones((4, 4, 4)), dirs, B=2, h=0.0)
