"""GPU test of vet_closure_noalloc, the entry point that allocates nothing.

Callers that cannot call cudaMalloc (another framework's allocator holds the
device memory, a real-time loop must not block on the allocator, or a host
application forbids allocations outside its own pool) use this entry point;
its workspace is a static device array inside libvet.  It must give what the
context path (vet_create + vet_closure) gives, on every call, although each
call reuses the array the previous call left behind.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from gpu_common import f_error, moment_errors
from paper_2202_08778_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2202_08778_gb300 import vet  # noqa: E402

FTOL32, RTOL32 = 1e-6, 1e-5  # the FP32 parity tolerances of the closure


def _problem(case):
    if case == "blob32":
        p = synth.blob_problem(n=32, B=8, nside=2, seed=1)
        Ib = None
    else:
        p = synth.lognormal_problem(n=64, B=16, nside=4, seed=7)
        Ib = np.random.default_rng(7).uniform(0, 0.2, (6, 192)).astype(np.float32)
    dev = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return p, dev(p["kappa"].astype(np.float32)), dev(p["S"].astype(np.float32)), dev(Ib)


@pytest.mark.parametrize("case", ["blob32", "lognormal64"])
def test_noalloc_matches_context_path_on_consecutive_calls(case):
    p, kappa, S, Ib = _problem(case)
    n = kappa.numel()
    ctx = vet.Context(p["kappa"].shape, p["B"], p["h"], p["nside"], p["q"])
    f_ref = torch.empty(6 * n, device="cuda")
    M_ref = torch.empty(10 * n, device="cuda")
    ctx.closure(kappa, S, Ib, f_ref, M_ref)
    ctx.sync()
    f_ref = f_ref.cpu().numpy().reshape(6, -1)
    M_ref = M_ref.cpu().numpy().reshape(10, -1).astype(np.float64)
    for call in range(2):
        f = torch.full((6 * n,), float("nan"), device="cuda")
        M = torch.full((10 * n,), float("nan"), device="cuda") if call == 0 else None
        vet.closure_noalloc(p["kappa"].shape, p["B"], p["h"], p["nside"], kappa, S, Ib, f, M, rot_q=p["q"])
        torch.cuda.synchronize()
        f = f.cpu().numpy().reshape(6, -1)
        assert np.isfinite(f).all()
        assert f_error(f, f_ref, M_ref) <= FTOL32
        if M is not None:
            eE, eFP = moment_errors(M.cpu().numpy(), M_ref)
            assert eE <= RTOL32 and eFP <= RTOL32


def test_noalloc_rejects_problems_beyond_its_static_workspace():
    kappa = torch.zeros(128 ** 3, device="cuda")
    f = torch.empty(6 * 128 ** 3, device="cuda")
    with pytest.raises(vet.VetError) as err:
        vet.closure_noalloc((128, 128, 128), 16, 1 / 128, 4, kappa, kappa, None, f)
    assert err.value.status == vet.VET_EINVAL
    assert "bytes of workspace" in str(err.value)
