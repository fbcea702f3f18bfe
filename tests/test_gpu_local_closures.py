"""GPU parity of vet_local_closure (paper Sec. 4.1) against the FP64 oracle
(oracle/local_closures.py), on seeded moments that cover the reduced-flux
range [0, 1], clipped fluxes above E, zero flux, and E = 0 and E < 0, with
cell counts that take the 16-byte path (a multiple of 4) and the scalar one.

Tolerance: the kernel evaluates the factor and the tensor in FP32 from the
same FP32 moments the oracle reads in FP64; each component is a handful of
roundings of values of order 1 (|T_ij| <= 1), so 2e-6 absolute is about 16
ulp of 1.  A wrong component, coefficient or clipping moves them by O(0.1).
"""
import numpy as np
import pytest

from oracle import local_closures as lc

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2202_08778_gb300 import vet  # noqa: E402

TOL = 2e-6


def _moments(n, seed):
    rng = np.random.default_rng(seed)
    E = rng.lognormal(0.0, 2.0, n)
    d = rng.normal(size=(3, n))
    d /= np.linalg.norm(d, axis=0)
    f = rng.uniform(0.0, 1.2, n)           # above 1: clipped
    F = d * f * E
    M = np.zeros((10, n), dtype=np.float32)
    M[0] = E
    M[1:4] = F
    k = n // 20
    M[1:4, :k] = 0.0                        # no flux
    M[0, k:2 * k] = 0.0                     # no radiation
    M[0, 2 * k:3 * k] *= -1.0               # unphysical E < 0
    M[4:] = rng.normal(size=(6, n))         # P is not read
    return M


@pytest.mark.parametrize("n,seed", [(1 << 16, 1), (10007, 2), (5, 3)])
def test_m1_matches_oracle(n, seed):
    M = _moments(n, seed)
    T = torch.full((6 * n,), np.nan, dtype=torch.float32, device="cuda")
    vet.local_closure(vet.VET_CLOSURE_M1, torch.from_numpy(M.ravel()).cuda(), T, n)
    torch.cuda.synchronize()
    got = T.cpu().numpy().reshape(6, n)
    ref = lc.m1(M.astype(np.float64))
    err = np.abs(got - ref).max()
    print(f"M1 n={n}: max |dT| {err:.2e}")
    assert err < TOL
    assert np.abs(got[0] + got[1] + got[2] - 1.0).max() < 1e-6


def test_eddington_is_a_third():
    n = 1001
    T = torch.full((6 * n,), np.nan, dtype=torch.float32, device="cuda")
    vet.local_closure(vet.VET_CLOSURE_EDDINGTON, None, T, n)
    torch.cuda.synchronize()
    got = T.cpu().numpy().reshape(6, n)
    np.testing.assert_array_equal(got[:3], np.float32(1.0 / 3.0))
    np.testing.assert_array_equal(got[3:], 0.0)


def test_m1_of_traced_moments_agrees_with_vet_where_radiation_streams():
    """On the moments of a single beam in vacuum the ray-traced VET and M1
    agree (both give n n: the flux fixes the direction of a free-streaming
    field); a check of the layouts the two entry points share."""
    from paper_2202_08778_gb300 import synth

    p = synth.blob_problem(n=16, B=8, nside=2, seed=51)
    ctx = vet.Context(p["kappa"].shape, p["B"], p["h"], p["nside"], p["q"])
    Ib = np.zeros((6, ctx.N), dtype=np.float32)
    Ib[:, 29] = 1.0
    zero = torch.zeros(16 ** 3, dtype=torch.float32, device="cuda")
    f = torch.empty(6 * 16 ** 3, dtype=torch.float32, device="cuda")
    M = torch.empty(10 * 16 ** 3, dtype=torch.float32, device="cuda")
    ctx.closure(zero, zero, torch.from_numpy(Ib).cuda(), f, M)
    T = torch.empty_like(f)
    vet.local_closure(vet.VET_CLOSURE_M1, M, T)
    torch.cuda.synchronize()
    assert (T - f).abs().max().item() < 1e-5


def test_arguments_are_checked():
    T = torch.empty(6 * 8, dtype=torch.float32, device="cuda")
    with pytest.raises(vet.VetError):
        vet.local_closure(7, None, T, 8)
    with pytest.raises(vet.VetError):
        vet.local_closure(vet.VET_CLOSURE_M1, None, T, 8)
    with pytest.raises(vet.VetError):  # host output
        vet.local_closure(vet.VET_CLOSURE_EDDINGTON, None, np.empty(6 * 8, dtype=np.float32), 8)
