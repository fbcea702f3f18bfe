"""Batched closures of independent ragged grids (one CUDA graph, one branch
per grid): equal to the grids' own closures (bit for bit where those do not
split their cell pass's last wave), repeatable on graph replay,
within tolerance of the FP64 oracle, and unchanged (to rounding) by the
autotuner's choice of tiles."""
import numpy as np
import pytest

from gpu_common import f_error, moment_errors
from paper_2202_08778_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2202_08778_gb300 import vet  # noqa: E402


def _batch(problems):
    specs = [(p["kappa"].shape, p["B"], p["h"], p["nside"], p["q"]) for p in problems]
    k = [torch.from_numpy(p["kappa"].astype(np.float32)).cuda() for p in problems]
    s = [torch.from_numpy(p["S"].astype(np.float32)).cuda() for p in problems]
    return specs, k, s


def test_small_ragged_batch_matches_single_grids_and_oracle(ora):
    problems = synth.batched_problems(n_grids=6, seed0=100, edges=(16, 32, 48), blocks=(8, 16), nsides=(2, 4))
    specs, k, s = _batch(problems)
    batch = vet.Batch(specs)
    f = [torch.empty(6 * x.numel(), device="cuda") for x in k]
    M = [torch.empty(10 * x.numel(), device="cuda") for x in k]
    batch.closure(k, s, None, f, M)
    batch.sync()
    first = [x.clone() for x in f]
    batch.closure(k, s, None, f, M)  # graph replay
    batch.sync()
    for i, p in enumerate(problems):
        assert torch.equal(f[i], first[i])
        ctx = vet.Context(*specs[i])
        fr = torch.empty_like(f[i])
        Mr = torch.empty_like(M[i])
        ctx.closure(k[i], s[i], None, fr, Mr)
        ctx.sync()
        assert torch.equal(fr, f[i]) and torch.equal(Mr, M[i])
    small = sorted(range(len(problems)), key=lambda i: problems[i]["kappa"].size)[:2]
    for i in small:
        p = problems[i]
        kk = p["kappa"].astype(np.float32).astype(np.float64)
        ss = p["S"].astype(np.float32).astype(np.float64)
        f_ref, M_ref, _, _ = ora.vet_closure(kk, ss, batch.members[i].directions(), p["B"], p["h"])
        eE, eFP = moment_errors(M[i].cpu().numpy(), M_ref)
        assert eE < 1e-5 and eFP < 1e-5
        assert f_error(f[i].cpu().numpy(), f_ref, M_ref) < 1e-6


def test_autotune_keeps_results_and_picks_valid_tiles():
    problems = synth.batched_problems(n_grids=4, seed0=120, edges=(32, 48), blocks=(8, 16), nsides=(2, 4))
    specs, k, s = _batch(problems)
    batch = vet.Batch(specs)
    f0 = [torch.empty(6 * x.numel(), device="cuda") for x in k]
    batch.closure(k, s, None, f0)
    batch.sync()
    batch.autotune(k, s)
    for m in batch.members:
        fg, dt = m.tuning()
        assert fg in (2, 4, 8) and dt in (1, 2, 3, 4, 5, 6, 7, 8)
    f1 = [torch.empty_like(x) for x in f0]
    batch.closure(k, s, None, f1)
    batch.sync()
    for a, b in zip(f0, f1):
        assert (a - b).abs().max().item() < 1e-6


def test_config4_batch_of_64_ragged_grids(ora):
    """The 64-grid batch (edges 32..96, 8^3 or 16^3 blocks, 48 or 192
    directions): every grid against the FP64 oracle on every cell (2.4e9
    cell-angles, about 40 s on 16 host cores), and four grids against their
    own closures (to rounding: a lone grid of more than one wave of cell-pass
    CTAs splits its last wave's work by directions, a batch member does not,
    so the sums are added in another order)."""
    problems = synth.batched_problems(n_grids=64, seed0=100)
    specs, k, s = _batch(problems)
    batch = vet.Batch(specs)
    f = [torch.empty(6 * x.numel(), device="cuda") for x in k]
    M = [torch.empty(10 * x.numel(), device="cuda") for x in k]
    batch.closure(k, s, None, f, M)
    batch.sync()
    for i in (0, 17, 42, 63):
        ctx = vet.Context(*specs[i])
        fr = torch.empty_like(f[i])
        ctx.closure(k[i], s[i], None, fr)
        ctx.sync()
        assert (fr - f[i]).abs().max().item() < 1e-6, i
    worst = (0.0, 0.0, 0.0)
    for i, p in enumerate(problems):
        kk = p["kappa"].astype(np.float32).astype(np.float64)
        ss = p["S"].astype(np.float32).astype(np.float64)
        f_ref, M_ref, _, _ = ora.vet_closure(kk, ss, batch.members[i].directions(), p["B"], p["h"])
        eE, eFP = moment_errors(M[i].cpu().numpy(), M_ref)
        ef = f_error(f[i].cpu().numpy(), f_ref, M_ref)
        assert eE < 1e-5 and eFP < 1e-5 and ef < 1e-6, (i, p["kappa"].shape, p["B"], p["nside"], eE, eFP, ef)
        worst = tuple(max(a, b) for a, b in zip(worst, (eE, eFP, ef)))
    print(f"64 ragged grids against the oracle: E rel {worst[0]:.2e}, F/P rel {worst[1]:.2e}, max |df| {worst[2]:.2e}")


def test_retuning_a_member_recaptures_the_batch_graph():
    """A member retuned through the batch (a new face-pass schedule, whose old
    item list the captured graph would read after it was freed, and a new
    cell-pass tile) must make the next batched closure capture again: its
    results then equal the grids' own closures at the new tuning."""
    problems = synth.batched_problems(n_grids=3, seed0=140, edges=(32, 48), blocks=(16,), nsides=(4,))
    specs, k, s = _batch(problems)
    batch = vet.Batch(specs)
    f = [torch.empty(6 * x.numel(), device="cuda") for x in k]
    batch.closure(k, s, None, f)
    batch.sync()
    fg0, dt0 = batch.members[0].tuning()
    batch.members[0].set_tuning(face_group=2 if fg0 != 2 else 8, dir_tile=4 if dt0 != 4 else 2)
    assert batch.members[0].tuning() != (fg0, dt0)
    batch.closure(k, s, None, f)
    batch.sync()
    for i in range(len(problems)):
        ctx = vet.Context(*specs[i])
        ctx.set_tuning(*batch.members[i].tuning())
        fr = torch.empty_like(f[i])
        ctx.closure(k[i], s[i], None, fr)
        ctx.sync()
        assert torch.equal(fr, f[i]), i
