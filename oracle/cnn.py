"""FP64 CPU oracle of the learned closure (TEST INFRASTRUCTURE ONLY).

The learned closure is not in the VETTAM paper; its definition here follows
the project's specification of it (a 3D convolutional network mapping local
features of kappa, S and E to the Eddington tensor, with the exact ray tracer
as fallback) and is written in plain numpy so that a reader can check every
step:

  features  -- per cell: validity mask, log10 of the cell optical depth
               kappa h, log10 S and log10 E (each minus its grid mean: f does
               not change when S, hence I and E, is scaled), and the mean and
               standard deviation of the log optical depth over the cell's
               block, broadcast to its cells;
  conv3d    -- 3x3x3 cross-correlation with zero padding ("same"):
               out[o, c] = b[o] + sum_taps sum_i W[tap, o, i] x[i, c + tap];
               tap = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
  network   -- conv(6 -> C) SiLU, conv(C -> C) SiLU, conv(C -> C) SiLU,
               conv(C -> 7); SiLU(z) = z / (1 + exp(-z));
  head      -- outputs 0..5 are a correction D to the isotropic tensor in the
               order xx, yy, zz, xy, xz, yz; the trace is projected out:
               f_ii = 1/3 + D_ii - (D_xx + D_yy + D_zz)/3, f_ij = D_ij;
               output 6 is the log of the predicted error, e = exp(o6);
  loss      -- mean over cells and the 6 components of (f - f_ref)^2 plus
               lam * mean over cells of (o6 - log(max_ij |f - f_ref| + 1e-4))^2
               (the error target is treated as a constant);
  indicator -- r = max(max(0, -lambda_min(f)), max(0, lambda_max(f) - 1), e).

Parity: pinned by finite differences of the loss (backward), one-hot kernels
(forward), and closed forms of the head and the eigenvalues.
"""
from __future__ import annotations

import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
N_IN, N_OUT = 6, 7
ERR_EPS = 1e-4


def features(kappa, S, E, h, B):
    """[6][nz][ny][nx] features of a grid (FP64)."""
    kappa = np.asarray(kappa, np.float64)
    tau = np.log10(np.maximum(kappa * h, 1e-30))
    ls = np.log10(np.maximum(np.asarray(S, np.float64), 1e-30))
    le = np.log10(np.maximum(np.asarray(E, np.float64), 1e-30))
    nz, ny, nx = kappa.shape
    blocks = tau.reshape(nz // B, B, ny // B, B, nx // B, B)
    mean = blocks.mean(axis=(1, 3, 5))
    std = blocks.std(axis=(1, 3, 5))
    up = lambda a: np.repeat(np.repeat(np.repeat(a, B, 0), B, 1), B, 2)
    return np.stack([np.ones_like(tau), tau, ls - ls.mean(), le - le.mean(), up(mean), up(std)])


def conv3d(x, W, b):
    """x [Cin][Z][Y][X], W [27][Cout][Cin], b [Cout] -> [Cout][Z][Y][X]."""
    cin, Z, Y, X = x.shape
    xp = np.zeros((cin, Z + 2, Y + 2, X + 2))
    xp[:, 1:-1, 1:-1, 1:-1] = x
    out = np.broadcast_to(np.asarray(b, np.float64)[:, None, None, None], (W.shape[1], Z, Y, X)).copy()
    for t, (dz, dy, dx) in enumerate(TAPS):
        sh = xp[:, 1 + dz:1 + dz + Z, 1 + dy:1 + dy + Y, 1 + dx:1 + dx + X]
        out += np.einsum("oi,izyx->ozyx", W[t], sh)
    return out


def conv3d_backward(x, W, gout):
    """Gradients of sum(gout * conv3d(x, W, b)) w.r.t. x, W and b."""
    cin, Z, Y, X = x.shape
    xp = np.zeros((cin, Z + 2, Y + 2, X + 2))
    xp[:, 1:-1, 1:-1, 1:-1] = x
    gxp = np.zeros_like(xp)
    gW = np.zeros_like(W)
    for t, (dz, dy, dx) in enumerate(TAPS):
        sl = (slice(None), slice(1 + dz, 1 + dz + Z), slice(1 + dy, 1 + dy + Y), slice(1 + dx, 1 + dx + X))
        gW[t] = np.einsum("ozyx,izyx->oi", gout, xp[sl])
        gxp[sl] += np.einsum("oi,ozyx->izyx", W[t], gout)
    return gxp[:, 1:-1, 1:-1, 1:-1], gW, gout.sum(axis=(1, 2, 3))


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def init_params(channels=32, seed=0):
    """He-style uniform initialisation; the last layer starts at zero (the
    network starts as the isotropic closure with a constant error guess)."""
    rng = np.random.default_rng(seed)
    shapes = [(N_IN, channels), (channels, channels), (channels, channels), (channels, N_OUT)]
    params = []
    for li, (ci, co) in enumerate(shapes):
        bound = np.sqrt(6.0 / (27 * ci))
        W = rng.uniform(-bound, bound, (27, co, ci)) if li < 3 else np.zeros((27, co, ci))
        b = np.zeros(co)
        if li == 3:
            b[6] = np.log(1e-2)
        params.append((W, b))
    return params


def forward(params, feat):
    """Returns (outputs [7][...], cache)."""
    acts, pres = [feat], []
    x = feat
    for li, (W, b) in enumerate(params):
        z = conv3d(x, W, b)
        pres.append(z)
        x = silu(z) if li < 3 else z
        acts.append(x)
    return x, (acts, pres)


def head(o):
    """(f [6][...], log-error o6) from outputs."""
    D = o[:6]
    tr = (D[0] + D[1] + D[2]) / 3.0
    f = D.copy()
    f[:3] = 1.0 / 3.0 + D[:3] - tr
    return f, o[6]


def error_target(o, f_ref):
    """log(max_ij |f - f_ref| + 1e-4): the regression target of output 6."""
    f, _ = head(o)
    return np.log(np.max(np.abs(f - f_ref), axis=0) + ERR_EPS)


def loss_and_grad_outputs(o, f_ref, lam=0.01, mask=None, tgt=None):
    """Loss and its gradient w.r.t. the outputs.  mask [...] selects the
    cells that count (all when None); the error target is a constant of the
    gradient (computed from o unless given)."""
    f, le = head(o)
    m = np.ones(f.shape[1:]) if mask is None else mask.astype(np.float64)
    n = m.sum()
    diff = (f - f_ref) * m
    if tgt is None:
        tgt = error_target(o, f_ref)
    r = (le - tgt) * m
    loss = (diff ** 2).sum() / (6 * n) + lam * (r ** 2).sum() / n
    gf = 2.0 * diff / (6 * n)
    go = np.zeros_like(o)
    go[:6] = gf
    trace_g = (gf[0] + gf[1] + gf[2]) / 3.0
    go[:3] = gf[:3] - trace_g
    go[6] = lam * 2.0 * r / n
    return loss, go


def backward(params, cache, gout):
    """Parameter gradients [(gW, gb)] for output gradient gout."""
    acts, pres = cache
    grads = [None] * len(params)
    g = gout
    for li in range(len(params) - 1, -1, -1):
        if li < 3:
            g = g * silu_grad(pres[li])
        gx, gW, gb = conv3d_backward(acts[li], params[li][0], g)
        grads[li] = (gW, gb)
        g = gx
    return grads


def sym_eigs(f):
    """Eigenvalues (ascending) of the symmetric tensors f [6][...]."""
    T = np.stack([np.stack([f[0], f[3], f[4]], -1), np.stack([f[3], f[1], f[5]], -1),
                  np.stack([f[4], f[5], f[2]], -1)], -2)
    return np.linalg.eigvalsh(T)


def indicator(o):
    f, le = head(o)
    ev = sym_eigs(f)
    return np.maximum(np.maximum(np.maximum(0.0, -ev[..., 0]), np.maximum(0.0, ev[..., 2] - 1.0)), np.exp(le))


def adamw(param, grad, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, wd=1e-4):
    """One AdamW step (Loshchilov & Hutter 2019): decoupled weight decay."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    param = param - lr * (mh / (np.sqrt(vh) + eps) + wd * param)
    return param, m, v
