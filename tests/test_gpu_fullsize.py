"""GPU parity at the benchmark's full sizes, in the launch configuration
bench.py times.

- 128^3 lognormal workload (16^3 blocks, 192 directions): f, E, F, P on every
  cell against the FP64 oracle (the oracle traces all 192 directions over the
  full grid on the host cores, a few seconds).
- 256x128x128 shadow workload (16^3 blocks, 768 directions, beam through
  x = 0): I on every cell for a sample of directions (lit, grazing and
  shadowed) against the oracle's trace of the same directions; f checked by
  the properties that hold at any size (trace 1, eigenvalues in [0, 1]) and the
  shadow behind the cloud.
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


def test_lognormal128_every_cell_matches_oracle(ora):
    p = synth.lognormal_problem(n=128, B=16, nside=4, seed=2)
    ctx = vet.Context(p["kappa"].shape, p["B"], p["h"], p["nside"], p["q"])
    k = p["kappa"].astype(np.float32)
    s = p["S"].astype(np.float32)
    n = k.size
    f = torch.empty(6 * n, device="cuda")
    M = torch.empty(10 * n, device="cuda")
    ctx.closure(torch.from_numpy(k).cuda(), torch.from_numpy(s).cuda(), None, f, M)
    ctx.sync()
    f_ref, M_ref, _, _ = ora.vet_closure(k.astype(np.float64), s.astype(np.float64), ctx.directions(), p["B"], p["h"])
    eE, eFP = moment_errors(M.cpu().numpy(), M_ref)
    ef = f_error(f.cpu().numpy(), f_ref, M_ref)
    print(f"lognormal128 every cell: E rel {eE:.2e}, F/P rel {eFP:.2e}, max |df| {ef:.2e}")
    assert eE < RTOL32 and eFP < RTOL32, (eE, eFP)
    assert ef < FTOL32


def test_cloud_sampled_directions_and_shadow(ora):
    p = synth.cloud_problem(nx=256, ny=128, nz=128, B=16, nside=8, seed=3)
    ctx = vet.Context(p["kappa"].shape, p["B"], p["h"], p["nside"], p["q"])
    dirs = ctx.directions()
    Ib = synth.beam_ib(dirs, p["beam_half_angle_deg"]).astype(np.float32)
    lit = np.flatnonzero(Ib[0] > 0)
    assert 4 <= lit.size <= 7
    k = torch.from_numpy(p["kappa"].astype(np.float32)).cuda()
    s = torch.from_numpy(p["S"].astype(np.float32)).cuda()
    ib = torch.from_numpy(Ib).cuda()
    n = k.numel()
    rng = np.random.default_rng(3)
    sample = np.unique(np.concatenate([lit, rng.choice(dirs.shape[0], 8, replace=False)]))
    I = torch.empty(ctx.N * n, device="cuda")
    ctx.trace(k, s, ib, I)
    ctx.sync()
    I_gpu = I.view(ctx.N, n)[torch.from_numpy(sample).cuda()].cpu().numpy()
    del I
    I_ref = ora.trace(p["kappa"].astype(np.float32).astype(np.float64), p["S"], dirs[sample], p["B"], p["h"],
                      Ib[:, sample].astype(np.float64))
    assert rel_err(I_gpu, I_ref.reshape(sample.size, -1)) < RTOL32
    # closure: properties at full size
    f = torch.empty(6 * n, device="cuda")
    M = torch.empty(10 * n, device="cuda")
    ctx.closure(k, s, ib, f, M)
    ctx.sync()
    f = f.cpu().numpy().reshape(6, 128, 128, 256)
    E = M[:n].cpu().numpy().reshape(128, 128, 256)
    assert np.abs(f[0] + f[1] + f[2] - 1).max() < 1e-6
    sub = np.random.default_rng(0).choice(n, 2000, replace=False)
    ff = f.reshape(6, -1)[:, sub]
    T = np.stack([np.stack([ff[0], ff[3], ff[4]], -1), np.stack([ff[3], ff[1], ff[5]], -1),
                  np.stack([ff[4], ff[5], ff[2]], -1)], -2)
    ev = np.linalg.eigvalsh(T)
    assert ev.min() > -1e-6 and ev.max() < 1 + 1e-6
    # shadow: just behind the cloud (x in [1.12, 1.2], on the axis) vs beside it
    behind = E[60:68, 60:68, 144:154].mean()
    beside = E[10:18, 10:18, 144:154].mean()
    assert behind < 1e-6 * beside
