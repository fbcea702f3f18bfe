"""GPU parity of vet_hlle_wavespeed (paper Sec. 2.2.3, App. A) against the
FP64 oracle (oracle/hlle.py): every face of ragged grids along all three
axes, including cells with no radiation along the axis (f_aa = 0) and
transparent cells (kappa = 0), and on the tensor of a traced closure.

Grids whose nx is a multiple of 4 run the kernel's 16-byte path, the others
(and arrays that are not 16-byte aligned) its scalar path; both are checked.

Tolerance: the FP32 path takes about ten roundings and approximations of a
few ulp each (the per-launch constant (10 h)^2 log2(e) / 4, its products
with kappa twice and with the hardware reciprocal of f_aa, the sum of the
two cells' halves, the thin-segment cubic (3.4e-7) or the hardware
exponential and reciprocal, the hardware square root and the product by c);
the correction's sensitivity to tau is at most 1/2 in relative terms, so
2e-6 relative bounds it."""
import numpy as np
import pytest

from oracle import hlle
from paper_2202_08778_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2202_08778_gb300 import vet  # noqa: E402

RTOL = 2e-6


def _offset(t, shift):
    """t on the device, starting `shift` floats into a larger buffer (shift
    1: 4 bytes past a 16-byte boundary)."""
    buf = torch.empty(t.numel() + shift, device="cuda")
    buf[shift:] = t.reshape(-1).cuda()
    return buf[shift:]


def _check(f32, k32, h, c=1.0, shift=0):
    nz, ny, nx = k32.shape
    fd = _offset(torch.from_numpy(np.ascontiguousarray(f32.reshape(-1))), shift)
    kd = _offset(torch.from_numpy(np.ascontiguousarray(k32.reshape(-1))), shift)
    worst = 0.0
    for axis in range(3):
        ext = [nz, ny, nx]
        ext[2 - axis] += 1
        C = _offset(torch.zeros(int(np.prod(ext))), shift)
        vet.hlle_wavespeed((nz, ny, nx), h, fd, kd, C, axis, c)
        torch.cuda.synchronize()
        got = C.cpu().numpy().reshape(ext)
        want = hlle.wavespeeds(f32.astype(np.float64), k32.astype(np.float64), float(np.float32(h)), axis, c)
        assert np.array_equal(got == 0.0, want == 0.0), axis
        nz_ = want != 0.0
        err = float((np.abs(got[nz_] - want[nz_]) / want[nz_]).max()) if nz_.any() else 0.0
        worst = max(worst, err)
    return worst


def _random_fields(rng, shape):
    f = np.zeros((6,) + shape, dtype=np.float32)
    f[:3] = rng.uniform(0.0, 1.0, (3,) + shape)
    f[:3] /= f[:3].sum(0)
    k = rng.lognormal(0.0, 2.5, shape).astype(np.float32)
    # degenerate cells: no radiation along an axis, transparent cells
    f[0].flat[:: 7] = 0.0
    f[1].flat[3:: 11] = 0.0
    k.flat[2:: 5] = 0.0
    return f, k


def test_random_tensors_on_ragged_grids():
    rng = np.random.default_rng(11)
    # nx 9 and 33: scalar path; 4, 12 and 8: 16-byte path with ragged ny, nz
    for shape in ((5, 7, 9), (16, 3, 33), (1, 1, 4), (3, 5, 12), (7, 1, 8)):
        f, k = _random_fields(rng, shape)
        err = _check(f, k, 1.0 / max(shape))
        print(f"hlle {shape}: max rel err {err:.2e}")
        assert err < RTOL


def test_unaligned_arrays_take_the_scalar_path():
    """nx a multiple of 4 but the arrays 4 bytes off a 16-byte boundary: the
    scalar path, with the same results as the aligned call."""
    rng = np.random.default_rng(12)
    f, k = _random_fields(rng, (4, 6, 16))
    err = _check(f, k, 1.0 / 16, shift=1)
    print(f"hlle unaligned: max rel err {err:.2e}")
    assert err < RTOL


def test_on_a_traced_closure():
    p = synth.blob_problem(n=16, B=8, nside=2, seed=1)
    ctx = vet.Context(p["kappa"].shape, p["B"], p["h"], p["nside"], p["q"])
    k = p["kappa"].astype(np.float32)
    s = p["S"].astype(np.float32)
    f = torch.empty(6 * k.size, device="cuda")
    ctx.closure(torch.from_numpy(k).cuda(), torch.from_numpy(s).cuda(), None, f)
    ctx.sync()
    err = _check(f.cpu().numpy().reshape((6,) + k.shape), k, p["h"], c=3.0)
    print(f"hlle on the blob closure: max rel err {err:.2e}")
    assert err < RTOL


def test_argument_errors():
    k = torch.ones(8, device="cuda")
    f = torch.ones(48, device="cuda")
    C = torch.empty(12, device="cuda")
    with pytest.raises(vet.VetError):
        vet.hlle_wavespeed((2, 2, 2), 0.5, f, k, C, 3)
    with pytest.raises(vet.VetError):
        vet.hlle_wavespeed((2, 2, 2), 0.5, f, k, torch.empty(12), 0)  # host output
    with pytest.raises(vet.VetError):
        vet.hlle_wavespeed((2, 2, 2), 0.5, f, k, C, 0, c=0.0)
