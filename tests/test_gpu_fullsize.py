"""GPU parity at the benchmark's full sizes, in the launch configuration
bench.py times.

- 128^3 lognormal workload (16^3 blocks, 192 directions): f, E, F, P on every
  cell against the FP64 oracle (the oracle traces all 192 directions over the
  full grid on the host cores, a few seconds).
- 256x128x128 shadow workload (16^3 blocks, 768 directions, beam through
  x = 0): S = 0 and the boundary is dark except for the beam's 4-7 directions,
  so every other direction's intensity is exactly 0 on both sides.  I on every
  cell and all 768 directions (the beam directions against the oracle's
  trace, the others checked to be 0 exactly), E, F, P and f on every cell
  against the oracle's moments and closure; f against the closed-form beam
  tensor in the lit streaming region; E in the deep shadow behind the cloud.
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


def test_cloud_every_cell_and_direction_matches_oracle(ora):
    p = synth.cloud_problem(nx=256, ny=128, nz=128, B=16, nside=8, seed=3)
    nx, ny, nz, h = 256, 128, 128, p["h"]
    ctx = vet.Context(p["kappa"].shape, p["B"], h, p["nside"], p["q"])
    dirs = ctx.directions()
    N = ctx.N
    Ib = synth.beam_ib(dirs, p["beam_half_angle_deg"]).astype(np.float32)
    beam = np.flatnonzero(Ib[0] > 0)
    assert 4 <= beam.size <= 7 and np.count_nonzero(Ib) == beam.size
    k32 = p["kappa"].astype(np.float32)
    k = torch.from_numpy(k32).cuda()
    s = torch.from_numpy(p["S"].astype(np.float32)).cuda()
    ib = torch.from_numpy(Ib).cuda()
    n = k.numel()
    # intensities of all 768 directions (12.9 GB on the device)
    I = torch.empty(N * n, device="cuda")
    ctx.trace(k, s, ib, I)
    ctx.sync()
    Iv = I.view(N, n)
    dark = np.setdiff1d(np.arange(N), beam)
    per_dir_max = torch.amax(Iv.abs(), dim=1).cpu().numpy()
    assert per_dir_max[dark].max() == 0.0  # no source, dark boundary: exactly 0
    I_gpu = Iv[torch.from_numpy(beam).cuda()].cpu().numpy()
    del I, Iv
    kk = k32.astype(np.float64)
    I_ref = ora.trace(kk, p["S"], dirs[beam], p["B"], h, Ib[:, beam].astype(np.float64)).reshape(beam.size, -1)
    eI = rel_err(I_gpu, I_ref)
    # moments and f: the dark directions add exactly 0 on both sides
    M_ref = ora.moments(I_ref, dirs[beam])
    f_ref, _ = ora.closure(M_ref)
    f = torch.empty(6 * n, device="cuda")
    M = torch.empty(10 * n, device="cuda")
    ctx.closure(k, s, ib, f, M)
    ctx.sync()
    f = f.cpu().numpy().reshape(6, -1)
    M = M.cpu().numpy().reshape(10, -1)
    eE, eFP = moment_errors(M, M_ref)
    ef = f_error(f, f_ref, M_ref)
    print(f"cloud 256x128x128, 768 directions, every cell: I rel {eI:.2e}, E rel {eE:.2e}, F/P rel {eFP:.2e}, "
          f"max |df| {ef:.2e}")
    assert eI < RTOL32 and eE < RTOL32 and eFP < RTOL32, (eI, eE, eFP)
    assert ef < FTOL32, ef
    # lit streaming region (x < 0.5, 0.2 < y, z < 0.8: uniform ambient
    # opacity upstream, the beam's rays meet the x = 0 face): the field of
    # every beam direction is I_b exp(-kappa x / n_x), invariant in y and z,
    # so hybrid characteristics are exact and f is the beam tensor
    # sum_b w_b I_b n_b n_b / sum_b w_b I_b in closed form
    xc = (np.arange(nx) + 0.5) * h
    lx = xc < 0.5
    ly = np.abs((np.arange(ny) + 0.5) * h - 0.5) < 0.3
    region = (ly[:, None, None] & ly[None, :, None] & lx[None, None, :]).ravel()  # [z][y][x]
    kap = float(k32[0, 0, 0])
    nb = dirs[beam, :3]
    wt = dirs[beam, 3][:, None] * np.exp(-kap * xc[None, :] / nb[:, 0:1])  # [beam][x]
    pairs = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))
    f_cf = np.stack([(wt * (nb[:, a] * nb[:, b])[:, None]).sum(0) / wt.sum(0) for a, b in pairs])  # [6][x]
    ix = np.tile(np.arange(nx), ny * nz)[region]
    d_lit = np.abs(f[:, region] - f_cf[:, ix]).max()
    print(f"lit streaming region ({region.sum()} cells): max |f - beam tensor| {d_lit:.2e}")
    assert d_lit < FTOL32
    # deep shadow just behind the cloud (x in [1.12, 1.25], within 2 cells of
    # the axis): every beam ray crosses the cloud core (the oracle gives 1.5e-18)
    E = M[0].reshape(nz, ny, nx)
    E_lit = E[:, :, : int(0.5 / h)].max()
    behind = E[62:66, 62:66, int(1.12 / h): int(1.25 / h)].max()
    print(f"deep shadow: max E / E_lit = {behind / E_lit:.2e}")
    assert behind < 1e-12 * E_lit
