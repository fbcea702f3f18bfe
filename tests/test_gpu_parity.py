"""GPU parity: libvet (through its C ABI) against the FP64 CPU oracle,
element by element on seeded inputs.

Tolerances (FP32 path): relative 1e-5 on I, E, F, P (F and P measured
against E of the same cell) and absolute 1e-6 on f_ij, the figures the
closure is specified to hold.  The FP64 path is held to 1e-11 relative on I
and 1e-12 absolute on f: it differs from the oracle only in rounding order.
"""
import numpy as np
import pytest

from gpu_common import f_error, moment_errors, rel_err
from paper_2202_08778_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2202_08778_gb300 import vet  # noqa: E402

RTOL32, FTOL32 = 1e-5, 1e-6
RTOL64, FTOL64 = 1e-11, 1e-12


def _ctx(p, precision):
    return vet.Context(p["kappa"].shape, p["B"], p["h"], p["nside"], p["q"], precision=precision)


def _inputs(p, dtype, Ib=None):
    """Device tensors of kappa, S, Ib and the float64 copies of exactly the
    values the device sees (so input rounding is not counted as error)."""
    k = p["kappa"].astype(dtype)
    s = p["S"].astype(dtype)
    ib = None if Ib is None else np.ascontiguousarray(Ib.astype(dtype))
    dev = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return (dev(k), dev(s), dev(ib)), (k.astype(np.float64), s.astype(np.float64),
                                       None if ib is None else ib.astype(np.float64))


def _gpu_closure(ctx, dev_in, ncell, dtype):
    td = torch.float64 if dtype == np.float64 else torch.float32
    f = torch.empty(6 * ncell, dtype=td, device="cuda")
    M = torch.empty(10 * ncell, dtype=td, device="cuda")
    ctx.closure(dev_in[0], dev_in[1], dev_in[2], f, M)
    ctx.sync()
    return f.cpu().numpy().reshape(6, -1), M.cpu().numpy().reshape(10, -1)


def _gpu_trace(ctx, dev_in, ncell, dtype):
    td = torch.float64 if dtype == np.float64 else torch.float32
    I = torch.empty(ctx.N * ncell, dtype=td, device="cuda")
    ctx.trace(dev_in[0], dev_in[1], dev_in[2], I)
    ctx.sync()
    return I.cpu().numpy().reshape(ctx.N, -1)


def test_directions_match_oracle(ora):
    for nside, seed in ((1, None), (2, 3), (4, 4), (8, 5)):
        q = synth.IDENTITY_Q if seed is None else synth.rotation_quaternion(seed)
        ctx = vet.Context((8, 8, 8), 8, 0.1, nside, q)
        np.testing.assert_allclose(ctx.directions(), ora.healpix(nside, q), rtol=0, atol=2e-15)


@pytest.mark.parametrize("shape,B,nside", [((32, 32, 32), 8, 2), ((48, 32, 16), 16, 4), ((12, 12, 12), 4, 1)])
def test_work_counts_match_oracle(ora, shape, B, nside):
    q = synth.rotation_quaternion(nside)
    ctx = vet.Context(shape, B, 0.1, nside, q)
    assert ctx.work_counts() == ora.count_segments(shape, B, ora.healpix(nside, q))


# --------------------------------------------------------------- FP64 path
@pytest.mark.parametrize("case", ["blob32", "ragged", "single_block", "unrotated"])
def test_fp64_trace_and_closure_match_oracle(ora, case):
    if case == "blob32":
        p = synth.blob_problem(n=32, B=8, nside=2, seed=1)
        Ib = None
    elif case == "ragged":
        p = synth.lognormal_problem(shape=(8, 16, 24), B=8, nside=2, seed=12)
        Ib = np.random.default_rng(12).uniform(0, 0.3, (6, 48))
    elif case == "single_block":
        p = synth.lognormal_problem(shape=(16, 16, 16), B=16, nside=2, seed=13)
        Ib = np.random.default_rng(13).uniform(0, 0.3, (6, 48))
    else:
        p = synth.blob_problem(n=16, B=4, nside=1, seed=1, rotate=False)
        Ib = np.random.default_rng(14).uniform(0, 0.3, (6, 12))
    ctx = _ctx(p, vet.VET_FP64)
    dev_in, host_in = _inputs(p, np.float64, Ib)
    dirs = ctx.directions()
    f_ref, M_ref, I_ref, _ = ora.vet_closure(host_in[0], host_in[1], dirs, p["B"], p["h"], host_in[2])
    I = _gpu_trace(ctx, dev_in, I_ref[0].size, np.float64)
    assert rel_err(I, I_ref.reshape(ctx.N, -1)) < RTOL64
    f, M = _gpu_closure(ctx, dev_in, I_ref[0].size, np.float64)
    eE, eFP = moment_errors(M, M_ref)
    assert eE < RTOL64 and eFP < RTOL64
    assert f_error(f, f_ref, M_ref) < FTOL64


# --------------------------------------------------------------- FP32 path
# a rotation that takes one nside = 8 direction to |n_y| = 6.4e-6: its exits
# through y planes lie far beyond any block, and the mirrored passes must not
# let the never-read exit-table rows for them decide whether a pair mirrors
NEAR_PLANE_Q = np.array([np.sqrt(0.5), 1 / np.sqrt(10.0), 1 / np.sqrt(3.0), 0.2])


@pytest.mark.parametrize("case", ["blob32", "lognormal48", "cloud", "ragged", "tiny_blocks", "unrotated8",
                                  "unrotated16", "near_plane8", "near_plane16", "single_block16", "vacuum",
                                  "opaque", "block12", "tail_split"])
def test_fp32_closure_matches_oracle(ora, case):
    """The unrotated cases hold directions with an exactly zero component (the
    HEALPix equator ring, n_z = 0), where a direction and its antipode both
    count the zero axis as positive: the paired cell pass must then take the
    in-plane face coordinates of each ray from its own direction, and the
    face pass runs unpaired."""
    Ib = None
    if case.startswith("near_plane"):
        B = 8 if case == "near_plane8" else 16
        p = synth.lognormal_problem(shape=(16, 16, 32), B=B, nside=8, seed=26)
        p["q"] = NEAR_PLANE_Q / np.linalg.norm(NEAR_PLANE_Q)
        Ib = np.random.default_rng(26).uniform(0, 0.5, (6, 768))
    elif case == "unrotated8":
        p = synth.blob_problem(n=16, B=8, nside=2, seed=1, rotate=False)
        Ib = np.random.default_rng(24).uniform(0, 0.5, (6, 48))
    elif case == "unrotated16":
        p = synth.lognormal_problem(n=32, B=16, nside=4, seed=25, rotate=False)
        Ib = np.random.default_rng(25).uniform(0, 0.5, (6, 192))
    elif case == "blob32":
        p = synth.blob_problem(n=32, B=8, nside=2, seed=1)
    elif case == "lognormal48":
        p = synth.lognormal_problem(n=48, B=16, nside=4, seed=2)
    elif case == "cloud":
        p = synth.cloud_problem(nx=64, ny=32, nz=32, B=16, nside=4, seed=3)
    elif case == "single_block16":  # one block: no face-pass level, every entry from the boundary
        p = synth.lognormal_problem(n=16, B=16, nside=4, seed=27)
        Ib = np.random.default_rng(27).uniform(0, 0.5, (6, 192))
    elif case == "vacuum":  # kappa = 0: every ray carries its boundary value unchanged
        p = synth.lognormal_problem(shape=(16, 32, 48), B=16, nside=4, seed=28)
        p["kappa"] = np.zeros_like(p["kappa"])
        Ib = np.random.default_rng(28).uniform(0, 0.5, (6, 192))
    elif case == "opaque":  # 1e4 optical depths per cell: I = S to rounding
        p = synth.lognormal_problem(n=32, B=8, nside=2, seed=29)
        p["kappa"] = np.full_like(p["kappa"], 1e4 / p["h"])
        Ib = np.random.default_rng(29).uniform(0, 0.5, (6, 48))
    elif case == "tail_split":  # 256 paired cell-pass CTAs: the last partial wave runs as direction shares
        p = synth.lognormal_problem(shape=(64, 64, 128), B=16, nside=4, seed=31)
        Ib = np.random.default_rng(31).uniform(0, 0.5, (6, 192))
    elif case == "block12":  # a block edge the mirrored kernels do not take (generic passes)
        p = synth.lognormal_problem(shape=(24, 36, 48), B=12, nside=2, seed=30)
    elif case == "ragged":
        p = synth.lognormal_problem(shape=(24, 16, 40), B=8, nside=2, seed=22)
        Ib = np.random.default_rng(22).uniform(0, 0.5, (6, 48))
    else:
        p = synth.lognormal_problem(shape=(6, 10, 8), B=2, nside=1, seed=23)
        Ib = np.random.default_rng(23).uniform(0, 0.5, (6, 12))
    ctx = _ctx(p, vet.VET_FP32)
    dirs = ctx.directions()
    if case == "cloud":
        Ib = synth.beam_ib(dirs, p["beam_half_angle_deg"])
    dev_in, host_in = _inputs(p, np.float32, Ib)
    f_ref, M_ref, I_ref, _ = ora.vet_closure(host_in[0], host_in[1], dirs, p["B"], p["h"], host_in[2])
    I = _gpu_trace(ctx, dev_in, I_ref[0].size, np.float32)
    assert rel_err(I, I_ref.reshape(ctx.N, -1)) < RTOL32
    if case == "opaque":  # the last half cell alone is 5e3 optical depths: I is the cell's S exactly
        assert np.array_equal(I, np.broadcast_to(host_in[1].astype(np.float32).ravel(), I.shape))
    f, M = _gpu_closure(ctx, dev_in, I_ref[0].size, np.float32)
    eE, eFP = moment_errors(M, M_ref)
    assert eE < RTOL32 and eFP < RTOL32, (eE, eFP)
    assert f_error(f, f_ref, M_ref) < FTOL32


@pytest.mark.parametrize("seed", [101, 102, 103, 104, 105, 106])
def test_fp32_closure_matches_oracle_on_random_rotations(ora, seed):
    """Haar-random rotations of the nside = 4 set: whichever direction pairs
    the host finds to be exact mirrors run paired, the others ray by ray."""
    B = 8 if seed % 2 else 16
    p = synth.lognormal_problem(shape=(16, 32, 32), B=B, nside=4, seed=seed)
    Ib = np.random.default_rng(seed).uniform(0, 0.5, (6, 192))
    ctx = _ctx(p, vet.VET_FP32)
    dev_in, host_in = _inputs(p, np.float32, Ib)
    f_ref, M_ref, _, _ = ora.vet_closure(host_in[0], host_in[1], ctx.directions(), p["B"], p["h"], host_in[2])
    f, M = _gpu_closure(ctx, dev_in, f_ref[0].size, np.float32)
    eE, eFP = moment_errors(M, M_ref)
    assert eE < RTOL32 and eFP < RTOL32, (eE, eFP)
    assert f_error(f, f_ref, M_ref) < FTOL32


def test_fp32_moments_entry_point_matches_oracle(ora):
    p = synth.lognormal_problem(n=16, B=8, nside=2, seed=31)
    ctx = _ctx(p, vet.VET_FP32)
    rng = np.random.default_rng(31)
    I = rng.lognormal(0.0, 1.0, (ctx.N, 16 ** 3)).astype(np.float32)
    M = torch.empty(10 * 16 ** 3, dtype=torch.float32, device="cuda")
    ctx.moments(torch.from_numpy(I).cuda(), M)
    ctx.sync()
    M_ref = ora.moments(I.astype(np.float64), ctx.directions())
    eE, eFP = moment_errors(M.cpu().numpy(), M_ref)
    assert eE < 1e-6 and eFP < 1e-6
    # the optional FP64 E: the oracle's FP64 E of the same FP32 intensities,
    # to FP64 rounding (the sum of 48 values), not FP32's
    E64 = torch.full((16 ** 3,), -1.0, dtype=torch.float64, device="cuda")
    ctx.moments(torch.from_numpy(I).cuda(), M, E64_out=E64)
    ctx.sync()
    e64 = E64.cpu().numpy()
    assert np.abs(e64 - M_ref[0].ravel()).max() / M_ref[0].max() < 1e-14
    with pytest.raises(vet.VetError):  # a host E64_out is refused
        ctx.moments(torch.from_numpy(I).cuda(), M, E64_out=torch.zeros(16 ** 3, dtype=torch.float64))


def test_host_buffers_give_identical_results():
    p = synth.blob_problem(n=32, B=8, nside=2, seed=1)
    ctx = _ctx(p, vet.VET_FP32)
    dev_in, _ = _inputs(p, np.float32)
    f_dev, M_dev = _gpu_closure(ctx, dev_in, 32 ** 3, np.float32)
    k = p["kappa"].astype(np.float32)
    s = p["S"].astype(np.float32)
    f_host = np.empty(6 * 32 ** 3, dtype=np.float32)
    M_host = np.empty(10 * 32 ** 3, dtype=np.float32)
    ctx.closure(k, s, None, f_host, M_host)
    np.testing.assert_array_equal(f_host.reshape(6, -1), f_dev)
    np.testing.assert_array_equal(M_host.reshape(10, -1), M_dev)


def test_pinned_host_outputs_are_written_in_place():
    """Outputs in pinned host memory are written by the kernels directly; the
    call returns only once they are complete, with device inputs too."""
    p = synth.blob_problem(n=32, B=8, nside=2, seed=1)
    ctx = _ctx(p, vet.VET_FP32)
    dev_in, _ = _inputs(p, np.float32)
    f_dev, M_dev = _gpu_closure(ctx, dev_in, 32 ** 3, np.float32)
    for inputs in ((dev_in[0], dev_in[1]), (dev_in[0].cpu().pin_memory(), dev_in[1].cpu().pin_memory())):
        f_pin = torch.full((6 * 32 ** 3,), np.nan, dtype=torch.float32).pin_memory()
        M_pin = torch.full((10 * 32 ** 3,), np.nan, dtype=torch.float32).pin_memory()
        ctx.closure(inputs[0], inputs[1], None, f_pin, M_pin)
        np.testing.assert_array_equal(f_pin.numpy().reshape(6, -1), f_dev)
        np.testing.assert_array_equal(M_pin.numpy().reshape(10, -1), M_dev)
    I_dev = _gpu_trace(ctx, dev_in, 32 ** 3, np.float32)
    I_pin = torch.full((ctx.N * 32 ** 3,), np.nan, dtype=torch.float32).pin_memory()
    ctx.trace(dev_in[0], dev_in[1], None, I_pin)
    np.testing.assert_array_equal(I_pin.numpy().reshape(ctx.N, -1), I_dev)


def test_repeat_runs_are_bit_identical():
    p = synth.lognormal_problem(n=32, B=16, nside=2, seed=41)
    ctx = _ctx(p, vet.VET_FP32)
    dev_in, _ = _inputs(p, np.float32)
    a = _gpu_closure(ctx, dev_in, 32 ** 3, np.float32)
    b = _gpu_closure(ctx, dev_in, 32 ** 3, np.float32)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_beam_in_vacuum_gives_n_outer_n_on_gpu():
    p = synth.blob_problem(n=16, B=8, nside=2, seed=51)
    ctx = _ctx(p, vet.VET_FP32)
    k0 = 29
    Ib = np.zeros((6, ctx.N), dtype=np.float32)
    Ib[:, k0] = 1.0
    zero = torch.zeros(16 ** 3, dtype=torch.float32, device="cuda")
    f = torch.empty(6 * 16 ** 3, dtype=torch.float32, device="cuda")
    ctx.closure(zero, zero, torch.from_numpy(Ib).cuda(), f)
    ctx.sync()
    n = ctx.directions()[k0, :3]
    want = [n[0] * n[0], n[1] * n[1], n[2] * n[2], n[0] * n[1], n[0] * n[2], n[1] * n[2]]
    got = f.cpu().numpy().reshape(6, -1)
    for m in range(6):
        assert np.abs(got[m] - want[m]).max() < 1e-6


def test_no_radiation_gives_isotropic_tensor():
    ctx = vet.Context((8, 8, 8), 4, 0.1, 1, synth.rotation_quaternion(1))
    zero = torch.zeros(512, dtype=torch.float32, device="cuda")
    f = torch.empty(6 * 512, dtype=torch.float32, device="cuda")
    ctx.closure(zero, zero, None, f)
    ctx.sync()
    got = f.cpu().numpy().reshape(6, -1)
    np.testing.assert_array_equal(got[:3], np.float32(1.0 / 3.0))
    np.testing.assert_array_equal(got[3:], 0.0)


def test_argument_errors_are_reported():
    ctx = vet.Context((8, 8, 8), 4, 0.1, 1)
    t = torch.zeros(512, dtype=torch.float32, device="cuda")
    with pytest.raises(vet.VetError):
        ctx.closure(None, t, None, torch.empty(6 * 512, device="cuda"))
    with pytest.raises(ValueError):
        ctx.closure(t, t, None, torch.empty(5 * 512, device="cuda"))
    lib = vet.load()
    assert lib.vet_trace_f64(ctx._h, t.data_ptr(), t.data_ptr(), None, t.data_ptr(), None) == vet.VET_EINVAL
    for bad in (dict(shape=(8, 8, 9), block=4), dict(shape=(8, 8, 8), block=1), dict(shape=(8, 8, 8), block=4, nside=3)):
        kw = dict(h=0.1, nside=1)
        kw.update(bad)
        with pytest.raises(vet.VetError):
            vet.Context(kw.pop("shape"), kw.pop("block"), **kw)
