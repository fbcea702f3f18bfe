"""Pins for the FP64 oracle of the learned closure (oracle/cnn.py): one-hot
kernels, finite differences, closed forms.  No expected value here comes from
the oracle itself."""
import numpy as np
import pytest

from oracle import cnn


def _rng(s):
    return np.random.default_rng(s)


def test_conv3d_one_hot_kernel_is_a_zero_padded_shift():
    rng = _rng(1)
    x = rng.standard_normal((3, 4, 5, 6))
    for t, (dz, dy, dx) in [(0, cnn.TAPS[0]), (13, cnn.TAPS[13]), (26, cnn.TAPS[26]), (7, cnn.TAPS[7])]:
        W = np.zeros((27, 2, 3))
        W[t, 1, 2] = 1.0
        out = cnn.conv3d(x, W, np.array([0.5, -1.0]))
        want = np.zeros((4, 5, 6))
        for z in range(4):
            for y in range(5):
                for xx in range(6):
                    zz, yy, xs = z + dz, y + dy, xx + dx
                    if 0 <= zz < 4 and 0 <= yy < 5 and 0 <= xs < 6:
                        want[z, y, xx] = x[2, zz, yy, xs]
        np.testing.assert_array_equal(out[0], 0.5)
        np.testing.assert_allclose(out[1], want - 1.0, atol=1e-15)


def test_conv3d_backward_matches_finite_differences():
    rng = _rng(2)
    x = rng.standard_normal((3, 4, 4, 5))
    W = rng.standard_normal((27, 2, 3))
    b = rng.standard_normal(2)
    g = rng.standard_normal((2, 4, 4, 5))
    gx, gW, gb = cnn.conv3d_backward(x, W, g)
    L = lambda x_, W_, b_: (g * cnn.conv3d(x_, W_, b_)).sum()
    eps = 1e-6
    for idx in [(0, 0, 0, 0), (2, 3, 1, 4), (1, 2, 2, 2)]:
        d = np.zeros_like(x)
        d[idx] = eps
        assert abs((L(x + d, W, b) - L(x - d, W, b)) / (2 * eps) - gx[idx]) < 1e-7
    for idx in [(0, 0, 0), (13, 1, 2), (26, 0, 1)]:
        d = np.zeros_like(W)
        d[idx] = eps
        assert abs((L(x, W + d, b) - L(x, W - d, b)) / (2 * eps) - gW[idx]) < 1e-7
    np.testing.assert_allclose(gb, g.sum(axis=(1, 2, 3)))


def test_head_is_trace_one_and_isotropic_at_zero():
    rng = _rng(3)
    o = rng.standard_normal((7, 3, 3, 3))
    f, le = cnn.head(o)
    np.testing.assert_allclose(f[0] + f[1] + f[2], 1.0, atol=1e-15)
    np.testing.assert_array_equal(f[3:], o[3:6])
    f0, _ = cnn.head(np.zeros((7, 2)))
    np.testing.assert_allclose(f0[:3], 1.0 / 3.0)
    np.testing.assert_array_equal(f0[3:], 0.0)


def test_network_gradient_matches_finite_differences():
    rng = _rng(4)
    params = cnn.init_params(channels=4, seed=4)
    params = [(W + 0.05 * rng.standard_normal(W.shape), b + 0.05 * rng.standard_normal(b.shape)) for W, b in params]
    feat = rng.standard_normal((6, 5, 4, 4))
    f_ref = rng.uniform(-0.2, 0.5, (6, 5, 4, 4))
    mask = np.ones((5, 4, 4), bool)
    mask[0] = False

    o, cache = cnn.forward(params, feat)
    tgt = cnn.error_target(o, f_ref)  # a constant of the gradient

    def loss(ps):
        oo, _ = cnn.forward(ps, feat)
        return cnn.loss_and_grad_outputs(oo, f_ref, lam=0.05, mask=mask, tgt=tgt)[0]

    _, go = cnn.loss_and_grad_outputs(o, f_ref, lam=0.05, mask=mask, tgt=tgt)
    grads = cnn.backward(params, cache, go)
    eps = 1e-6
    for li, idx in [(0, (13, 1, 2)), (1, (0, 3, 3)), (2, (26, 0, 1)), (3, (13, 6, 2)), (3, (5, 0, 3))]:
        W, b = params[li]
        ps_p = [(w.copy(), bb.copy()) for w, bb in params]
        ps_m = [(w.copy(), bb.copy()) for w, bb in params]
        ps_p[li][0][idx] += eps
        ps_m[li][0][idx] -= eps
        fd = (loss(ps_p) - loss(ps_m)) / (2 * eps)
        assert abs(fd - grads[li][0][idx]) < 1e-6 * max(1.0, abs(fd)), (li, idx, fd, grads[li][0][idx])
    for li in range(4):
        ps_p = [(w.copy(), bb.copy()) for w, bb in params]
        ps_m = [(w.copy(), bb.copy()) for w, bb in params]
        ps_p[li][1][0] += eps
        ps_m[li][1][0] -= eps
        fd = (loss(ps_p) - loss(ps_m)) / (2 * eps)
        assert abs(fd - grads[li][1][0]) < 1e-6 * max(1.0, abs(fd))


def test_eigenvalues_and_indicator_closed_forms():
    f = np.zeros((6, 3))
    f[:3, 0] = [0.5, 0.3, 0.2]          # diagonal: eigenvalues are the entries
    f[:3, 1] = [1 / 3, 1 / 3, 1 / 3]
    f[0, 2], f[1, 2], f[3, 2] = 0.5, 0.5, 0.5  # [[.5,.5,0],[.5,.5,0],[0,0,0]]: 0, 0, 1
    ev = cnn.sym_eigs(f)
    np.testing.assert_allclose(ev[0], [0.2, 0.3, 0.5])
    np.testing.assert_allclose(ev[1], [1 / 3] * 3)
    np.testing.assert_allclose(ev[2], [0.0, 0.0, 1.0], atol=1e-15)
    o = np.zeros((7, 2))
    o[6] = np.log([1e-3, 5e-2])
    o[3, 1] = 0.6  # xy = 0.6 with diagonal 1/3: eigenvalues 1/3 +- 0.6
    r = cnn.indicator(o)
    assert abs(r[0] - 1e-3) < 1e-15
    assert abs(r[1] - (0.6 - 1 / 3)) < 1e-12


def test_features_block_stats_and_scale_invariance():
    rng = _rng(5)
    kappa = np.exp(rng.standard_normal((8, 8, 8)))
    S = np.exp(rng.standard_normal((8, 8, 8)))
    E = np.exp(rng.standard_normal((8, 8, 8)))
    f1 = cnn.features(kappa, S, E, h=0.1, B=4)
    f2 = cnn.features(kappa, 7.0 * S, 3.0 * E, h=0.1, B=4)
    np.testing.assert_allclose(f1, f2, atol=1e-12)
    np.testing.assert_array_equal(f1[0], 1.0)
    tau = np.log10(kappa * 0.1)
    np.testing.assert_allclose(f1[4][0, 0, 0], tau[:4, :4, :4].mean())
    np.testing.assert_allclose(f1[5][7, 7, 7], tau[4:, 4:, 4:].std())
    const = cnn.features(np.full((4, 4, 4), 2.0), np.ones((4, 4, 4)), np.ones((4, 4, 4)), h=0.5, B=4)
    np.testing.assert_allclose(const[4], 0.0, atol=1e-15)
    np.testing.assert_allclose(const[5], 0.0, atol=1e-15)


def test_adamw_first_step_moves_by_learning_rate():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([3.0, -0.1, 0.0])
    p1, m, v = cnn.adamw(p, g, np.zeros(3), np.zeros(3), step=1, lr=0.01, wd=0.0)
    # first bias-corrected step is lr * g / (|g| + eps)
    np.testing.assert_allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8))
    p2, _, _ = cnn.adamw(p, np.zeros(3), np.zeros(3), np.zeros(3), step=1, lr=0.01, wd=0.1)
    np.testing.assert_allclose(p2, p * (1 - 0.01 * 0.1))
