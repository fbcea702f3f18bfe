"""Failure detection on the GPU without a fault: every device-side wait of
the closure (a CTA waiting for its TMA-staged data, or for its warps to
release a buffer) is bounded by the context's spin_limit.  With a limit of one
poll the waits give up; the call must then report VET_ETIMEOUT through
vet_sync, and the device and the library must stay usable."""
import numpy as np
import pytest

from paper_2202_08778_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2202_08778_gb300 import vet  # noqa: E402


def test_bounded_waits_report_timeout_and_context_stays_usable():
    p = synth.lognormal_problem(n=64, B=16, nside=4, seed=5)
    k = torch.from_numpy(p["kappa"].astype(np.float32)).cuda()
    s = torch.from_numpy(p["S"].astype(np.float32)).cuda()
    n = k.numel()
    good = vet.Context(p["kappa"].shape, p["B"], p["h"], p["nside"], p["q"])
    f_ref = torch.empty(6 * n, device="cuda")
    good.closure(k, s, None, f_ref)
    good.sync()
    impatient = vet.Context(p["kappa"].shape, p["B"], p["h"], p["nside"], p["q"], spin_limit=1)
    f = torch.empty(6 * n, device="cuda")
    impatient.closure(k, s, None, f)
    with pytest.raises(vet.VetError) as err:
        impatient.sync()
    assert err.value.status == vet.VET_ETIMEOUT
    # the status was cleared and the device still answers: the patient context
    # repeats its result bit for bit
    f2 = torch.empty(6 * n, device="cuda")
    good.closure(k, s, None, f2)
    good.sync()
    assert torch.equal(f2, f_ref)
    assert torch.cuda.synchronize() is None
