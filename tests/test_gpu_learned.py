"""GPU parity of the learned closure: libvet's BF16 network kernels (through
the C ABI) against the FP64 oracle (oracle/cnn.py), its optimiser against
AdamW's first-step identity, its indicator against closed forms, and the
trained network plus exact fallback against the ray-traced closure.

Tolerances.  The kernels round features, weights and activations to BF16
(8 significant bits, relative rounding error <= 2^-9 = 2e-3 per value) and
accumulate in FP32.  Weights are rounded to BF16 on the host before both sides
see them, so the differences left are the BF16 rounding of the 6 input
features, of the three hidden activations and (backward) of the propagated
gradients.  Each output sums 27 x C_in such terms with independent rounding
errors, so the relative error of a sum is about 2^-9 / sqrt(27 C_in) ~ 1e-4
per layer, not 2^-9: measured on GB300, the forward pass is within 3.0e-4 of
the largest output (RMS 1.9e-4 of the RMS output), the loss within 1.1e-5
relative and every layer's gradient within 1.3e-4 in relative Frobenius norm.
The bounds below are about 6x those figures: a wrong tap, channel or sign
moves them by O(1).
"""
import math

import numpy as np
import pytest

from oracle import cnn
from paper_2202_08778_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2202_08778_gb300 import vet  # noqa: E402


def bf16_round(a):
    """Round float32 values to the nearest BF16 value (ties to even)."""
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def _params(seed, last_scale=0.3, bias_scale=0.1):
    """He-initialised layers (oracle.cnn.init_params) with a random last layer
    and biases, rounded to BF16 so both sides use the same numbers."""
    rng = np.random.default_rng(seed)
    ps = cnn.init_params(32, seed=seed)
    out = []
    for li, (W, b) in enumerate(ps):
        if li == 3:
            W = rng.uniform(-1, 1, W.shape) * last_scale * math.sqrt(6.0 / (27 * 32))
        b = b + bias_scale * rng.standard_normal(b.shape)
        out.append((bf16_round(W).astype(np.float64), np.float32(b).astype(np.float64)))
    return out


def _fields(rng, nvol, shape):
    """Lognormal kappa, S, E of nvol volumes: [nvol][nz][ny][nx] float32."""
    kappa = np.exp(rng.normal(2.0, 1.5, (nvol, *shape))).astype(np.float32)
    S = np.exp(rng.normal(0.0, 1.0, (nvol, *shape))).astype(np.float32)
    E = np.exp(rng.normal(1.0, 1.0, (nvol, *shape))).astype(np.float32)
    return kappa, S, E


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


SHAPE, B, H, NVOL = (10, 12, 20), 2, 1.0 / 20, 2  # ragged in every tile dimension (8 x 8 x 4 tiles)


def test_features_match_oracle():
    rng = np.random.default_rng(11)
    kappa, S, E = _fields(rng, NVOL, SHAPE)
    m = vet.Model()
    n = NVOL * int(np.prod(SHAPE))
    feat = torch.empty(6 * n, device="cuda")
    m.features(SHAPE, B, H, _dev(kappa), _dev(S), _dev(E), nvol=NVOL, feat_out=feat)
    got = feat.cpu().numpy().reshape(NVOL, 6, *SHAPE)
    for v in range(NVOL):
        ref = cnn.features(kappa[v], S[v], E[v], H, B)
        err = np.abs(got[v] - ref).max()
        print(f"features volume {v}: max abs error {err:.2e}")
        assert err < 2e-5


def _oracle_forward(params, kappa, S, E):
    outs, caches = [], []
    for v in range(kappa.shape[0]):
        o, cache = cnn.forward(params, cnn.features(kappa[v], S[v], E[v], H, B))
        outs.append(o)
        caches.append(cache)
    return np.stack(outs, 1), caches  # [7][nvol][...]


def test_forward_matches_oracle():
    rng = np.random.default_rng(12)
    kappa, S, E = _fields(rng, NVOL, SHAPE)
    params = _params(12)
    m = vet.Model()
    m.set_params(params)
    n = NVOL * int(np.prod(SHAPE))
    o = torch.empty(7 * n, device="cuda")
    m.features(SHAPE, B, H, _dev(kappa), _dev(S), _dev(E), nvol=NVOL)
    m.forward(o)
    got = o.cpu().numpy().reshape(NVOL, 7, *SHAPE).transpose(1, 0, 2, 3, 4)
    ref, _ = _oracle_forward(params, kappa, S, E)
    scale = np.abs(ref).max()
    err = np.abs(got - ref)
    rms = math.sqrt((err ** 2).mean()) / math.sqrt((ref ** 2).mean())
    print(f"forward: max |o| {scale:.3f}, max error {err.max() / scale:.2e} of max, rms error {rms:.2e} of rms")
    assert err.max() < 2e-3 * scale
    assert rms < 1e-3


def test_backward_matches_oracle():
    rng = np.random.default_rng(13)
    kappa, S, E = _fields(rng, NVOL, SHAPE)
    params = _params(13)
    f_ref = rng.uniform(-0.1, 0.5, (NVOL, 6, *SHAPE)).astype(np.float32)
    mask = (rng.uniform(size=(NVOL, *SHAPE)) < 0.8).astype(np.uint8)
    lam = 0.05
    m = vet.Model()
    m.set_params(params)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    m.features(SHAPE, B, H, _dev(kappa), _dev(S), _dev(E), nvol=NVOL)
    m.forward()
    m.backward(_dev(f_ref), _dev(mask), lam=lam, loss_out=loss)
    g_gpu = m.grads()

    o, caches = _oracle_forward(params, kappa, S, E)
    fr = f_ref.transpose(1, 0, 2, 3, 4).astype(np.float64)
    L, go = cnn.loss_and_grad_outputs(o, fr, lam=lam, mask=mask.astype(bool))
    g_ref = None
    for v in range(NVOL):
        gv = cnn.backward(params, caches[v], go[:, v])
        g_ref = gv if g_ref is None else [(a + c, b + d) for (a, b), (c, d) in zip(g_ref, gv)]
    lg = float(loss.item())
    print(f"loss gpu {lg:.6e} oracle {L:.6e}")
    assert abs(lg - L) < 1e-4 * L
    for li, ((gw, gb), (rw, rb)) in enumerate(zip(g_gpu, g_ref)):
        a = np.concatenate([gw.ravel(), gb.ravel()]).astype(np.float64)
        r = np.concatenate([rw.ravel(), rb.ravel()])
        rel = np.linalg.norm(a - r) / np.linalg.norm(r)
        cos = a @ r / (np.linalg.norm(a) * np.linalg.norm(r))
        print(f"layer {li}: gradient rel error {rel:.2e}, cosine {cos:.6f}")
        assert rel < 1e-3 and cos > 0.99999


def test_adamw_first_step_identity():
    """From fresh moments, AdamW's first step moves every parameter by
    -lr (g / (|g| + eps) + wd p): bias correction cancels (1 - beta)."""
    rng = np.random.default_rng(14)
    kappa, S, E = _fields(rng, 1, (8, 8, 8))
    params = _params(14)
    f_ref = rng.uniform(-0.1, 0.5, (1, 6, 8, 8, 8)).astype(np.float32)
    m = vet.Model()
    m.set_params(params)
    m.features((8, 8, 8), 4, 0.125, _dev(kappa), _dev(S), _dev(E))
    m.forward()
    m.backward(_dev(f_ref), lam=0.01)
    g = m.grads()
    lr, wd, eps = 1e-3, 1e-2, 1e-8
    m.step(lr=lr, weight_decay=wd, eps=eps)
    p1 = m.params()
    for (W0, b0), (gw, gb), (W1, b1) in zip(params, g, p1):
        for x0, gx, x1 in ((W0, gw, W1), (b0, gb, b1)):
            x0 = x0.astype(np.float32).astype(np.float64)
            gx = gx.astype(np.float64)
            want = x0 - lr * (gx / (np.abs(gx) + eps) + wd * x0)
            # float32 arithmetic: a few ulp of the parameter plus of the step
            assert np.abs(x1 - want).max() < 1e-6 * (np.abs(x0).max() + lr)


def test_save_and_load_round_trip(tmp_path):
    """Parameters written by Model.save come back bit for bit in another
    model, whose forward pass then equals the first model's."""
    rng = np.random.default_rng(15)
    kappa, S, E = _fields(rng, 1, (8, 8, 8))
    a, b = vet.Model(), vet.Model()
    a.set_params(_params(15))
    a.save(tmp_path / "net.vetm")
    b.load(tmp_path / "net.vetm")
    for (Wa, ba), (Wb, bb) in zip(a.params(), b.params()):
        np.testing.assert_array_equal(Wa, Wb)
        np.testing.assert_array_equal(ba, bb)
    outs = []
    for m in (a, b):
        m.features((8, 8, 8), 4, 0.125, _dev(kappa), _dev(S), _dev(E))
        o = torch.empty(7 * 512, dtype=torch.float32, device="cuda")
        m.forward(o)
        torch.cuda.synchronize()
        outs.append(o.cpu().numpy())
    np.testing.assert_array_equal(outs[0], outs[1])
    # a file of another hidden width, a truncated file and a foreign file are
    # refused, and the model keeps its parameters
    raw = (tmp_path / "net.vetm").read_bytes()
    assert raw[:8] == b"VETMODL1" and int.from_bytes(raw[8:12], "little") == 32
    (tmp_path / "other.vetm").write_bytes(raw[:8] + (16).to_bytes(4, "little") + raw[12:])
    (tmp_path / "short.vetm").write_bytes(raw[: len(raw) // 2])
    (tmp_path / "foreign.vetm").write_bytes(b"NOTAMODEL" + raw[9:])
    for name in ("other.vetm", "short.vetm", "foreign.vetm"):
        with pytest.raises(vet.VetError):
            b.load(tmp_path / name)
    for (Wa, ba), (Wb, bb) in zip(a.params(), b.params()):
        np.testing.assert_array_equal(Wa, Wb)


def test_checkpoint_resumes_training(tmp_path):
    """Saving after some AdamW steps and loading into a fresh model carries
    the optimiser state and step count: the next step gives the same
    parameters in both models (to the rounding of the weight gradient's
    atomic sums), unlike a model given the parameters alone, whose AdamW
    restarts from zero moments."""
    rng = np.random.default_rng(16)
    kappa, S, E = _fields(rng, 1, (8, 8, 8))
    f_ref = _dev(rng.uniform(-0.1, 0.4, (6, 512)).astype(np.float32))
    a = vet.Model()
    a.set_params(_params(16))

    def train_step(m):
        m.features((8, 8, 8), 4, 0.125, _dev(kappa), _dev(S), _dev(E))
        m.forward()
        m.backward(f_ref, lam=0.01)
        m.step(lr=1e-3)

    for _ in range(3):
        train_step(a)
    a.save(tmp_path / "ckpt.vetm")
    b, c = vet.Model(), vet.Model()
    b.load(tmp_path / "ckpt.vetm")
    c.set_params(a.params())
    for m in (a, b, c):
        train_step(m)
    flat = lambda m: np.concatenate([np.concatenate([W.ravel(), bb.ravel()]) for W, bb in m.params()])
    pa, pb, pc = flat(a), flat(b), flat(c)
    assert np.abs(pa - pb).max() < 1e-6
    assert np.abs(pa - pc).max() > 1e-5


def test_indicator_closed_form_with_bias_only_network():
    """A network whose weights are zero outputs its last bias everywhere:
    f = head(b) and r = max(-lambda_min, lambda_max - 1, exp(b6)) are then
    closed forms (here f = I/3 + 0.6 (e_x e_y + e_y e_x) with eigenvalues
    1/3 - 0.6, 1/3, 1/3 + 0.6)."""
    shape, Bk = (16, 16, 16), 8
    ctx = vet.Context(shape, Bk, 1.0 / 16, 1)
    m = vet.Model()
    params = [(np.zeros((27, co, ci)), np.zeros(co)) for ci, co in vet.layer_shapes(32)]
    b = np.zeros(7)
    b[3] = 0.6
    b[6] = math.log(1e-3)
    params[3] = (params[3][0], b)
    m.set_params(params)
    rng = np.random.default_rng(15)
    kappa, S, E = (x[0] for x in _fields(rng, 1, shape))
    n = int(np.prod(shape))
    f = torch.empty(6 * n, device="cuda")
    r = torch.empty(n, device="cuda")
    flags = torch.zeros(8, dtype=torch.int32, device="cuda")
    nfb = m.closure(ctx, _dev(kappa), _dev(S), _dev(E), f, threshold=1.0, block_flags=flags)
    m.last_indicator(r, n)
    torch.cuda.synchronize()
    fn = f.cpu().numpy().reshape(6, -1)
    assert nfb == 0 and int(flags.sum()) == 0
    np.testing.assert_allclose(fn[:3], 1.0 / 3.0, atol=1e-7)
    np.testing.assert_allclose(fn[3], 0.6, atol=1e-7)
    np.testing.assert_array_equal(fn[4:], 0.0)
    np.testing.assert_allclose(r.cpu().numpy(), 0.6 - 1.0 / 3.0, rtol=1e-5)
    # the same network with a threshold below r: every block falls back to
    # the exact closure, so f equals vet_closure's f exactly
    nfb = m.closure(ctx, _dev(kappa), _dev(S), _dev(E), f, threshold=0.2, block_flags=flags)
    f_exact = torch.empty(6 * n, device="cuda")
    ctx.closure(_dev(kappa), _dev(S), None, f_exact)
    ctx.sync()
    assert nfb == 8 and int(flags.sum()) == 8
    assert torch.equal(f, f_exact)


# ----------------------------------------------------------------- training
TRAIN_SHAPE, TRAIN_B, NSIDE = (64, 64, 64), 16, 4


def _snapshots(seeds, ctx):
    """kappa, S, traced E and traced f of lognormal snapshots (device)."""
    n = int(np.prod(TRAIN_SHAPE))
    ks, ss, es, fs = [], [], [], []
    for s in seeds:
        p = synth.lognormal_problem(n=TRAIN_SHAPE[0], B=TRAIN_B, nside=NSIDE, seed=int(s))
        k = _dev(p["kappa"].astype(np.float32))
        S = _dev(p["S"].astype(np.float32))
        f = torch.empty(6 * n, device="cuda")
        M = torch.empty(10 * n, device="cuda")
        ctx.closure(k, S, None, f, M)
        ks.append(k)
        ss.append(S)
        es.append(M[:n].clone())
        fs.append(f)
    ctx.sync()
    return torch.stack(ks), torch.stack(ss), torch.stack(es), torch.stack(fs)


@pytest.fixture(scope="module")
def trained():
    ctx = vet.Context(TRAIN_SHAPE, TRAIN_B, 1.0 / TRAIN_SHAPE[0], NSIDE, synth.rotation_quaternion(10000))
    train = _snapshots(range(10000, 10016), ctx)
    held = _snapshots(range(20000, 20004), ctx)
    m = vet.Model()
    m.set_params(cnn.init_params(32, seed=0))
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    losses = []
    batch, steps = 2, 400
    rng = np.random.default_rng(0)
    for it in range(steps):
        idx = torch.from_numpy(rng.choice(len(train[0]), batch, replace=False)).cuda()
        k, S, E, f = (x.index_select(0, idx).contiguous() for x in train)
        m.features(TRAIN_SHAPE, TRAIN_B, 1.0 / TRAIN_SHAPE[0], k, S, E, nvol=batch)
        m.forward()
        m.backward(f, lam=2e-3, loss_out=loss)
        m.step(lr=2e-3 if it < 300 else 5e-4)
        if it % 50 == 0 or it == steps - 1:
            losses.append(float(loss.item()))
    print("training loss:", " ".join(f"{v:.3e}" for v in losses))
    return ctx, m, held, losses


def _net_f(m, k, S, E):
    n = int(np.prod(TRAIN_SHAPE))
    o = torch.empty(7 * n, device="cuda")
    m.features(TRAIN_SHAPE, TRAIN_B, 1.0 / TRAIN_SHAPE[0], k, S, E)
    m.forward(o)
    f, _ = cnn.head(o.cpu().numpy().reshape(7, -1).astype(np.float64))
    return f


def test_trained_network_beats_eddington(trained):
    ctx, m, held, losses = trained
    assert losses[-1] < 0.5 * losses[0]
    e_net, e_edd = [], []
    for v in range(held[0].shape[0]):
        f_ref = held[3][v].cpu().numpy().reshape(6, -1).astype(np.float64)
        f_net = _net_f(m, held[0][v], held[1][v], held[2][v])
        iso = np.zeros_like(f_ref)
        iso[:3] = 1.0 / 3.0
        e_net.append(np.sqrt(((f_net - f_ref) ** 2).mean()))
        e_edd.append(np.sqrt(((iso - f_ref) ** 2).mean()))
    print(f"held-out rms error: network {np.mean(e_net):.3e}, Eddington I/3 {np.mean(e_edd):.3e}")
    assert np.mean(e_net) < 0.7 * np.mean(e_edd)


def test_learned_closure_with_fallback(trained):
    ctx, m, held, _ = trained
    n = int(np.prod(TRAIN_SHAPE))
    nblk = n // TRAIN_B ** 3
    f = torch.empty(6 * n, device="cuda")
    flags = torch.zeros(nblk, dtype=torch.int32, device="cuda")
    f_plain = torch.empty(6 * n, device="cuda")
    kept = 0
    for v in range(held[0].shape[0]):
        k, S, E, f_tr = held[0][v], held[1][v], held[2][v], held[3][v]
        nfb = m.closure(ctx, k, S, E, f, threshold=1e-2, block_flags=flags)
        ctx.closure(k, S, None, f_plain)  # the same kernels as the fallback (no moments output)
        ctx.sync()
        fl = flags.cpu().numpy().astype(bool)
        assert fl.sum() == nfb
        got = f.cpu().numpy().reshape(6, *TRAIN_SHAPE)
        ref = f_plain.cpu().numpy().reshape(6, *TRAIN_SHAPE)
        assert np.abs(ref - f_tr.cpu().numpy().reshape(6, *TRAIN_SHAPE)).max() < 1e-6
        nb = TRAIN_SHAPE[0] // TRAIN_B
        blk = fl.reshape(nb, nb, nb)  # [bz][by][bx]
        cell_flag = np.repeat(np.repeat(np.repeat(blk, TRAIN_B, 0), TRAIN_B, 1), TRAIN_B, 2)
        # recomputed blocks equal the plain closure bit for bit
        assert np.array_equal(got[:, cell_flag], ref[:, cell_flag])
        err = np.abs(got - ref).max()
        print(f"held-out {v}: {nfb}/{nblk} blocks recomputed, max |f - f_traced| = {err:.3e}")
        # the accuracy contract: every block the network keeps is within 1e-2
        # of the traced tensor in every component
        assert err <= 1e-2, err
        kept += nblk - nfb
    # without fallback the result is the network's tensor everywhere
    nfb = m.closure(ctx, held[0][0], held[1][0], held[2][0], f, threshold=float("inf"), block_flags=flags)
    assert nfb == 0 and int(flags.sum()) == 0
    f_net = _net_f(m, held[0][0], held[1][0], held[2][0])
    assert np.abs(f.cpu().numpy().reshape(6, -1) - f_net).max() < 1e-6
    if kept == 0:
        pytest.xfail("the network kept no block at 1e-2 on the held-out fields: every block fell back to the "
                     "exact closure (the contract held trivially)")
