"""Training and evaluation helpers of the learned closure (the network and
its kernels are in libvet; see include/vet.h).

The training data are the method's own output: seeded lognormal snapshots
(synth.lognormal_problem) whose f and E come from the exact GPU closure.
Every step runs in libvet's kernels; this module only sequences the calls.
"""
from __future__ import annotations

import math

import numpy as np

from . import synth, vet


def init_params(channels: int = 32, seed: int = 0):
    """He-uniform weights (bound sqrt(6 / fan_in), fan_in = 27 C_in); the
    last layer starts at zero with the error output's bias at log(1e-2), so
    the untrained network is the isotropic closure I/3."""
    rng = np.random.default_rng(seed)
    out = []
    shapes = vet.layer_shapes(channels)
    for li, (ci, co) in enumerate(shapes):
        if li < len(shapes) - 1:
            bound = math.sqrt(6.0 / (27 * ci))
            W = rng.uniform(-bound, bound, (27, co, ci))
        else:
            W = np.zeros((27, co, ci))
        b = np.zeros(co)
        if li == len(shapes) - 1:
            b[6] = math.log(1e-2)
        out.append((W, b))
    return out


def snapshots(ctx, seeds, n: int, B: int, nside: int):
    """Device tensors (kappa, S, E, f) [len(seeds)][...] of lognormal n^3
    snapshots, labelled by the exact closure of ctx (same grid and
    directions)."""
    import torch

    N = n ** 3
    ks, ss, es, fs = [], [], [], []
    for s in seeds:
        p = synth.lognormal_problem(n=n, B=B, nside=nside, seed=int(s))
        k = torch.from_numpy(np.ascontiguousarray(p["kappa"].astype(np.float32))).cuda()
        S = torch.from_numpy(np.ascontiguousarray(p["S"].astype(np.float32))).cuda()
        f = torch.empty(6 * N, device="cuda")
        M = torch.empty(10 * N, device="cuda")
        ctx.closure(k, S, None, f, M)
        ks.append(k)
        ss.append(S)
        es.append(M[:N].clone())
        fs.append(f)
    ctx.sync()
    return tuple(torch.stack(x) for x in (ks, ss, es, fs))


def train(model, data, shape, B: int, h: float, steps: int, batch: int = 4, lr_max: float = 2e-3,
          lr_min: float = 1e-4, lam: float = 2e-3, seed: int = 0, log_every: int = 0):
    """AdamW with a cosine learning-rate schedule over random batches of the
    snapshots.  Returns the losses sampled every `log_every` steps (and the
    last one)."""
    import torch

    k_all, s_all, e_all, f_all = data
    n = k_all.shape[0]
    rng = np.random.default_rng(seed)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    losses = []
    for it in range(steps):
        idx = torch.from_numpy(rng.choice(n, batch, replace=False)).cuda()
        k, S, E, f = (x.index_select(0, idx).contiguous() for x in (k_all, s_all, e_all, f_all))
        model.features(shape, B, h, k, S, E, nvol=batch)
        model.forward()
        model.backward(f, lam=lam, loss_out=loss)
        lr = lr_min + 0.5 * (lr_max - lr_min) * (1.0 + math.cos(math.pi * it / steps))
        model.step(lr=lr)
        if (log_every and it % log_every == 0) or it == steps - 1:
            losses.append(float(loss.item()))
    return losses


def evaluate(model, data, shape, B: int, h: float, block_edge: int):
    """Held-out errors of the network's f against the traced f (per cell, the
    largest of the 6 components' absolute errors), of the Eddington tensor I/3
    for scale, and the fraction of blocks whose largest network error is
    below 1e-2.  data: (kappa, S, E, f) stacked as from snapshots()."""
    import torch

    k_all, s_all, e_all, f_all = data
    n = int(np.prod(shape))
    o = torch.empty(7 * n, device="cuda")
    e_net, e_edd, blocks_ok = [], [], []
    for v in range(k_all.shape[0]):
        model.features(shape, B, h, k_all[v], s_all[v], e_all[v])
        model.forward(o)
        D = o.view(7, -1)[:6].double()
        f = D.clone()
        tr = (D[0] + D[1] + D[2]) / 3.0
        f[:3] = 1.0 / 3.0 + D[:3] - tr
        ref = f_all[v].view(6, -1).double()
        err = (f - ref).abs().amax(0)
        iso = torch.zeros_like(ref)
        iso[:3] = 1.0 / 3.0
        e_net.append(err)
        e_edd.append((iso - ref).abs().amax(0))
        nb = [s_ // block_edge for s_ in shape]
        eb = err.view(nb[0], block_edge, nb[1], block_edge, nb[2], block_edge).amax(dim=(1, 3, 5))
        blocks_ok.append(float((eb < 1e-2).double().mean()))
    en, ee = torch.cat(e_net), torch.cat(e_edd)
    q = torch.quantile(en[::7], torch.tensor([0.5, 0.99], dtype=torch.float64, device=en.device))
    return {"net_mean": float(en.mean()), "net_p50": float(q[0]), "net_p99": float(q[1]), "net_max": float(en.max()),
            "eddington_mean": float(ee.mean()), "blocks_below_1e-2": float(np.mean(blocks_ok))}


def accepted_on_field(model, n: int = 256, B: int = 16, nside: int = 4, seed: int = 3, threshold: float = 1e-2):
    """The learned closure with fallback on a seeded n^3 lognormal field
    (E from the exact closure, as in the benchmark): blocks the indicator
    keeps, their largest |f - f_traced|, and the times of the plain and the
    learned closures (ms, medians of three)."""
    import statistics

    import torch

    p = synth.lognormal_problem(n=n, B=B, nside=nside, seed=seed)
    ctx = vet.Context(p["kappa"].shape, B, p["h"], nside, p["q"])
    k = torch.from_numpy(np.ascontiguousarray(p["kappa"].astype(np.float32))).cuda()
    S = torch.from_numpy(np.ascontiguousarray(p["S"].astype(np.float32))).cuda()
    N = n ** 3
    nblk = N // B ** 3
    f_plain = torch.empty(6 * N, device="cuda")
    M = torch.empty(10 * N, device="cuda")
    ctx.closure(k, S, None, f_plain, M)
    E = M[:N].clone()
    del M
    ctx.set_timing(True)
    plain = []
    for _ in range(3):
        ctx.closure(k, S, None, f_plain)
        plain.append(ctx.last_timing()[3])
    ctx.set_timing(False)
    f = torch.empty(6 * N, device="cuda")
    flags = torch.zeros(nblk, dtype=torch.int32, device="cuda")
    ts = []
    nfb = 0
    for _ in range(3):
        nfb = model.closure(ctx, k, S, E, f, threshold=threshold, block_flags=flags)
        ts.append(model.last_timing()[2])
    ctx.sync()
    kept = ~flags.bool()
    err = (f - f_plain).abs().view(6, -1).amax(0)
    nb = n // B
    eb = err.view(nb, B, nb, B, nb, B).amax(dim=(1, 3, 5)).reshape(-1)
    return {"blocks": nblk, "kept": int(kept.sum()), "kept_fraction": float(kept.double().mean()),
            "kept_max_abs_df": float(eb[kept].max()) if bool(kept.any()) else 0.0,
            "plain_ms": statistics.median(plain), "learned_ms": statistics.median(ts), "fallback_blocks": nfb}


def curve(counts=(64, 512, 2000), steps_per_snapshot: float = 10.0, min_steps: int = 1500, batch: int = 4,
          nt: int = 64, B: int = 16, nside: int = 4, lr_max: float = 2e-3):
    """Accuracy of the learned closure against the amount of training data:
    for each snapshot count, train from scratch on the first that many of
    2000 seeded 64^3 snapshots (seeds 10000..11999, labelled by the exact
    closure) and report held-out errors (16 snapshots, seeds 20000..20015)
    and the blocks the indicator keeps at 1e-2 on the 256^3 field of seed 3."""
    import time

    import torch

    ctx_t = vet.Context((nt,) * 3, B, 1.0 / nt, nside, synth.rotation_quaternion(10000))
    t0 = time.perf_counter()
    data = snapshots(ctx_t, range(10000, 10000 + max(counts)), nt, B, nside)
    held = snapshots(ctx_t, range(20000, 20016), nt, B, nside)
    t_data = time.perf_counter() - t0
    out = []
    for c in counts:
        sub = tuple(x[:c] for x in data)
        steps = max(min_steps, int(steps_per_snapshot * c))
        model = vet.Model()
        model.set_params(init_params(32, seed=0))
        t0 = time.perf_counter()
        losses = train(model, sub, (nt,) * 3, B, 1.0 / nt, steps, batch=batch, lr_max=lr_max)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        res = {"snapshots": c, "steps": steps, "batch": batch, "lr_max": lr_max, "train_seconds": t_train,
               "final_loss": losses[-1],
               "held_out": evaluate(model, held, (nt,) * 3, B, 1.0 / nt, B),
               "field256_seed3": accepted_on_field(model)}
        out.append(res)
        print(res, flush=True)
    return {"data_seconds": t_data, "runs": out}


def main(argv=None):
    """Without --train: run the learned closure (network only, no fallback) on
    a seeded n^3 lognormal field after the exact closure that supplies E and
    print the device timings (untrained network: cost, not accuracy).
    With --train: train the network on 64^3 snapshots of the lognormal
    generator labelled by the exact closure and print held-out errors.
    With --curve: the same for 64, 512 and 2000 snapshots, with the blocks
    the indicator keeps on the 256^3 field of seed 3 (one JSON line)."""
    import argparse
    import time

    import torch

    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--block", type=int, default=16)
    ap.add_argument("--nside", type=int, default=4)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--train", action="store_true")
    ap.add_argument("--snapshots", type=int, default=512)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--curve", action="store_true",
                    help="train on 64, 512 and 2000 snapshots and report errors and kept blocks")
    ap.add_argument("--counts", type=str, default="64,512,2000", help="snapshot counts of --curve")
    ap.add_argument("--lr", type=float, default=2e-3, help="peak learning rate of the cosine schedule (--curve)")
    a = ap.parse_args(argv)
    if a.curve:
        import json

        counts = tuple(int(c) for c in a.counts.split(","))
        print(json.dumps(curve(counts=counts, batch=a.batch, lr_max=a.lr)))
        return
    if a.train:
        nt = 64
        ctx_t = vet.Context((nt,) * 3, a.block, 1.0 / nt, a.nside, synth.rotation_quaternion(10000))
        t0 = time.perf_counter()
        data = snapshots(ctx_t, range(10000, 10000 + a.snapshots), nt, a.block, a.nside)
        held = snapshots(ctx_t, range(20000, 20016), nt, a.block, a.nside)
        t_data = time.perf_counter() - t0
        model = vet.Model()
        model.set_params(init_params(32, seed=0))
        t0 = time.perf_counter()
        losses = train(model, data, (nt,) * 3, a.block, 1.0 / nt, a.steps, batch=a.batch, log_every=max(1, a.steps // 10))
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        res = evaluate(model, held, (nt,) * 3, a.block, 1.0 / nt, a.block)
        print(f"data {t_data:.1f} s, training {t_train:.1f} s; loss " + " ".join(f"{v:.3e}" for v in losses))
        print("held-out (16 snapshots):", res)
        return
    p = synth.lognormal_problem(n=a.n, B=a.block, nside=a.nside, seed=a.seed)
    ctx = vet.Context(p["kappa"].shape, a.block, p["h"], a.nside, p["q"])
    k = torch.from_numpy(np.ascontiguousarray(p["kappa"].astype(np.float32))).cuda()
    S = torch.from_numpy(np.ascontiguousarray(p["S"].astype(np.float32))).cuda()
    N = a.n ** 3
    f = torch.empty(6 * N, device="cuda")
    M = torch.empty(10 * N, device="cuda")
    ctx.closure(k, S, None, f, M)
    ctx.sync()
    E = M[:N].clone()
    model = vet.Model()
    params = init_params(32, seed=0)
    W3, b3 = params[-1]
    params[-1] = (np.random.default_rng(0).uniform(-0.05, 0.05, W3.shape), b3)
    model.set_params(params)
    for _ in range(a.repeat):
        model.closure(ctx, k, S, E, f, threshold=float("inf"))
        print("learned closure ms (network, fallback, total, convolutions):", model.last_timing())


if __name__ == "__main__":
    main()
