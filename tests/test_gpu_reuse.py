"""GPU parity of the change gate (vet_field_change) and of the reuse of f
across time steps (paper Sec. 4.2) against the oracle (oracle/field_change.py).

The gate's numbers are FP32 with one IEEE rounding per operation and exact
maxima on both sides, so they are compared bit for bit: on ragged grids
with block edges that take the 16-byte path (multiples of 4) and the scalar
one, on fields that are not 16-byte aligned, with NaN, inf and negative
cells, and at the full 128^3 size in 16^3 blocks.  The reuse driver is
checked step by step on an advected lognormal sequence: its decisions equal
the oracle's decisions taken on the same numbers, a recomputed f equals a
fresh closure bit for bit, and a reused f is the stored one.
"""
import numpy as np
import pytest

from oracle import field_change as fc

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2202_08778_gb300 import synth, vet  # noqa: E402


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32).ravel()).cuda()


def _fields(shape, seed, specials=True):
    rng = np.random.default_rng(seed)
    k = rng.lognormal(2.0, 1.5, shape).astype(np.float32)
    s = rng.lognormal(0.0, 2.0, shape).astype(np.float32)
    kr = (k * rng.lognormal(0.0, 0.05, shape)).astype(np.float32)
    sr = (s * rng.lognormal(0.0, 0.05, shape)).astype(np.float32)
    same = rng.random(shape) < 0.3
    kr[same], sr[same] = k[same], s[same]
    if specials:
        flat = [a.reshape(-1) for a in (k, s, kr, sr)]
        n = k.size
        flat[0][n // 3] = np.nan
        flat[1][n // 2] = np.inf
        flat[3][n // 2] = np.inf
        flat[2][n // 5] = -3.0        # unphysical, still compared exactly
        flat[3][n - 1] = -2.5
    return k, s, kr, sr


def _gate(shape, B, h, k, s, kr, sr, snapshot=False, offset=0):
    n = k.size
    nb = n // B ** 3
    bufs = []
    for a in (k, s, kr, sr):
        t = torch.empty(n + offset, dtype=torch.float32, device="cuda")
        t[offset:] = _dev(a)
        bufs.append(t[offset:])
    out = torch.full((3 + 3 * nb,), np.nan, dtype=torch.float32, device="cuda")
    vet.field_change(shape, B, h, bufs[0], bufs[1], bufs[2], bufs[3], out, snapshot)
    torch.cuda.synchronize()
    return out.cpu().numpy(), [b.cpu().numpy() for b in bufs]


@pytest.mark.parametrize("shape,B,offset", [
    ((16, 24, 32), 8, 0),      # 16-byte path
    ((32, 16, 16), 16, 0),
    ((12, 18, 6), 6, 0),       # scalar path (edge not a multiple of 4)
    ((8, 8, 8), 2, 0),
    ((9, 9, 27), 3, 0),
    ((16, 8, 24), 4, 1),       # fields not 16-byte aligned: scalar path
    ((32, 32, 32), 32, 0),     # largest block edge
])
def test_gate_matches_oracle_bitwise(shape, B, offset):
    k, s, kr, sr = _fields(shape, 11 + B)
    h = 1.0 / 48
    got, _ = _gate(shape, B, h, k, s, kr, sr, offset=offset)
    ref = fc.change(k, s, kr, sr, h, B)
    np.testing.assert_array_equal(got, ref)


def test_snapshot_copies_the_fields_and_reports_the_change_before_it():
    shape, B, h = (16, 16, 24), 8, 0.05
    k, s, kr, sr = _fields(shape, 5, specials=False)
    got, bufs = _gate(shape, B, h, k, s, kr, sr, snapshot=True)
    np.testing.assert_array_equal(got, fc.change(k, s, kr, sr, h, B))
    np.testing.assert_array_equal(bufs[2], k.ravel())
    np.testing.assert_array_equal(bufs[3], s.ravel())
    got, _ = _gate(shape, B, h, k, s, k, s)
    assert np.all(got.reshape(-1, 3)[:, :2] == 0.0)


def test_gate_full_size_advected_lognormal():
    p, seq = synth.lognormal_sequence(n=128, B=16, nside=4, steps=2, cells_per_step=0.05)
    (k0, s0), (k1, s1) = seq
    got, _ = _gate(k0.shape, 16, p["h"], k1, s1, k0, s0)
    ref = fc.change(k1, s1, k0, s0, p["h"], 16)
    print(f"128^3 grid triple {got[:3]}")
    np.testing.assert_array_equal(got, ref)


def _fresh(ctx, k, s):
    f = torch.empty(6 * ctx.ncell, dtype=torch.float32, device="cuda")
    ctx.closure(_dev(k), _dev(s), None, f)
    torch.cuda.synchronize()
    return f.cpu().numpy()


@pytest.mark.parametrize("tol,max_age", [(0.05, 4), (0.2, 8), (0.0, 8)])
def test_reuse_follows_the_oracle_step_by_step(tol, max_age):
    p, seq = synth.lognormal_sequence(n=32, B=8, nside=2, steps=10, cells_per_step=0.01)
    ctx = vet.Context(p["kappa"].shape, p["B"], p["h"], p["nside"], p["q"])
    run = vet.ClosureReuse(ctx, tol_tau=tol, tol_S=tol, max_age=max_age)
    snap, stored, age, decisions = None, None, 0, []
    for t, (k, s) in enumerate(seq):
        f, redo = run.step(_dev(k), _dev(s))
        torch.cuda.synchronize()
        if snap is None:
            want = True
        else:
            ch = fc.change(k, s, snap[0], snap[1], p["h"], p["B"])
            np.testing.assert_array_equal(np.float32(run.last_change), ch[:3])
            want = fc.recompute(ch[:3], age, False, tol, tol, max_age)
        assert redo == want, (t, run.last_change)
        decisions.append(redo)
        if redo:
            snap, age = (k, s), 0
            stored = _fresh(ctx, k, s)
        else:
            age += 1
        np.testing.assert_array_equal(f.cpu().numpy(), stored)
    print(f"tol {tol}, max_age {max_age}: recomputed at steps {[i for i, d in enumerate(decisions) if d]}")
    assert run.recomputes == sum(decisions)
    if tol == 0.0:
        assert all(decisions)


def test_unchanged_fields_are_reused_until_max_age_and_force_recomputes():
    p = synth.blob_problem(n=16, B=8, nside=2, seed=3)
    ctx = vet.Context(p["kappa"].shape, p["B"], p["h"], p["nside"], p["q"])
    run = vet.ClosureReuse(ctx, max_age=3)
    k, s = _dev(p["kappa"]), _dev(p["S"])
    flags = [run.step(k, s)[1] for _ in range(8)]
    assert flags == [True, False, False, False, True, False, False, False]
    assert run.last_change[0] == 0.0 and run.last_change[1] == 0.0
    assert run.step(k, s, force=True)[1]
    np.testing.assert_array_equal(run.f.cpu().numpy(), _fresh(ctx, p["kappa"], p["S"]))


def test_arguments_are_checked():
    t = torch.zeros(64, dtype=torch.float32, device="cuda")
    out = torch.zeros(3 + 3 * 8, dtype=torch.float32, device="cuda")
    t6 = torch.zeros(96, dtype=torch.float32, device="cuda")
    with pytest.raises(vet.VetError):   # block edge does not divide the grid
        vet.field_change((4, 4, 6), 4, 0.1, t6, t6, t6.clone(), t6.clone(), out[:6])
    with pytest.raises(vet.VetError):   # host field
        vet.field_change((4, 4, 4), 2, 0.1, np.zeros(64, np.float32), t, t.clone(), t.clone(), out)
    with pytest.raises(vet.VetError):   # h <= 0
        vet.field_change((4, 4, 4), 2, 0.0, t, t, t.clone(), t.clone(), out)
