#!/usr/bin/env python
"""Throughput of the VET closure (VETTAM Sec. 2.2.5) on GB300.

One step = one full closure (face wavefront pass, cell pass with the
quadratures, f = P/E) over the 128^3 lognormal-opacity workload in 16^3
blocks with 192 HEALPix directions (nside = 4), inputs resident in HBM.
The metric is cell-angle updates per second (cells x directions / time) and
closures per second, at the accuracy the parity tests hold (|df| <= 1e-6
against the FP64 oracle).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

The line also carries, at N = 1, a "learned" object: the learned closure
(network + indicator + exact fallback on flagged blocks) at 256^3 against the
plain closure on the same GPU, with the network trained in the same run.

It also carries, at N = 1, a "batch" object: 64 ragged grids as one batched
closure (one CUDA graph) against the same closures launched one by one.

Prints one JSON line on rank 0.  With --gpus N > 1 (under torchrun) every
rank runs an independent replica of the workload on its own GPU (the method
has no data exchange between replicas); the value is the total over ranks
divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "G cell·angle updates/s and VET closures/s at fixed |Δf|≤1e-6 (plain) / ≤1e-2 (learned)"
UNIT = "G cell·angle updates/s"
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2
MUFU_PER_CLK_PER_SM = 32    # ex2 results per clock per SM on GB300 (csrc/peaks.cu measures 31.99)
N_SM = 152


def workload():
    from paper_2202_08778_gb300 import synth

    p = synth.lognormal_problem(n=128, B=16, nside=4, seed=2)
    return p, {"workload": "lognormal128_B16_nside4", "grid": [128, 128, 128], "block": 16, "n_dir": 192,
               "seed": 2, "boundary": "vacuum", "l2": "flushed between timed steps (256 MiB write)"}


def kernel_source_digest(paths) -> str:
    """SHA-256 of CUDA sources (one path or a list: the kernel's file and the
    headers that fix its constants and layouts) with comments and blank lines
    removed, so that a comment edit does not count as a kernel change."""
    import hashlib
    import re

    if isinstance(paths, str):
        paths = [paths]
    lines = []
    for path in paths:
        src = open(path, encoding="utf-8").read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        lines += [ln.rstrip() for ln in src.splitlines() if ln.strip()]
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()


def measured_traffic():
    """DRAM bytes per cell-pass launch from the committed ncu capture, or None
    if the kernel source changed since the counters were taken."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "cell_pass_lognormal128_traffic.json")))
        src = rec["source"] if isinstance(rec["source"], list) else [rec["source"]]
        digest = kernel_source_digest([os.path.join(ROOT, x) for x in src])
    except (OSError, ValueError, KeyError):
        return None
    if digest != rec.get("kernel_source_digest"):
        return None
    return rec.get("bytes_per_launch")


def slowest_rank_ms(total_ms: float, world: int, device=None) -> float:
    """The timed region's length over all ranks: the maximum of every rank's
    own total (one all-reduce; a barrier after it)."""
    if world <= 1:
        return total_ms
    import torch
    import torch.distributed as dist

    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, total_ms: float) -> float:
    """Units all ranks processed per second of the slowest rank's time."""
    return units_per_rank * world / (total_ms * 1e-3)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample(p, dirs, ndir_sample: int, Ib=None, grid_text: str = "128^3"):
    """Time the FP64 oracle (trace -> moments -> closure) on the workload's
    grid restricted to an evenly spaced subset of directions.  Returns
    (cell-angle updates per second, seconds, threads used, sample text)."""
    import numpy as np

    import oracle

    oracle.build()
    idx = np.linspace(0, dirs.shape[0] - 1, ndir_sample).round().astype(int)
    sub = dirs[idx].copy()
    cores = len(os.sched_getaffinity(0))
    k = p["kappa"].astype(np.float32).astype(np.float64)
    s = p["S"].astype(np.float32).astype(np.float64)
    ib = None if Ib is None else np.ascontiguousarray(Ib[:, idx], dtype=np.float64)
    t0 = time.perf_counter()
    I = oracle.trace(k, s, sub, p["B"], p["h"], ib, nthreads=cores)
    M = oracle.moments(I, sub)
    oracle.closure(M)
    dt = time.perf_counter() - t0
    upd = k.size * ndir_sample
    return upd / dt, dt, min(cores, ndir_sample), (
        f"{ndir_sample} of {dirs.shape[0]} directions (evenly spaced) over the full {grid_text} grid, "
        f"trace+moments+closure in FP64")


def workload_measurement(local_rank, kind: str, steps: int = 10, cpu: bool = True):
    """One of the two largest single-GPU workloads, timed like the headline
    (autotuned tiles, L2 flushed between steps, inputs in HBM): "shadow" is
    the 256x128x128 cloud in 16^3 blocks with 768 directions and the beam
    through x = 0; "lognormal256" the learned closure's 256^3 lognormal grid
    (16^3 blocks, 192 directions, seed 3) closed by the plain tracer.  With
    the cell-pass roofline, the closure through pinned host buffers and the
    FP64 oracle on a sample of directions over the full grid."""
    import numpy as np
    import torch

    from paper_2202_08778_gb300 import synth, vet

    dev = torch.device("cuda", local_rank)
    if kind == "shadow":
        p = synth.cloud_problem(nx=256, ny=128, nz=128, B=16, nside=8, seed=3)
        name, grid_text = "shadow256x128x128_B16_nside8 (beam within 10 deg of +x on x = 0)", "256x128x128"
    else:
        p = synth.lognormal_problem(n=256, B=16, nside=4, seed=3)
        name, grid_text = "lognormal256_B16_nside4 (seed 3)", "256^3"
    ctx = vet.Context(p["kappa"].shape, p["B"], p["h"], p["nside"], p["q"], device=local_rank)
    dirs = ctx.directions()
    Ib = synth.beam_ib(dirs, p["beam_half_angle_deg"]).astype(np.float32) if kind == "shadow" else None
    n, N = p["kappa"].size, ctx.N
    k_h = np.ascontiguousarray(p["kappa"].astype(np.float32))
    s_h = np.ascontiguousarray(p["S"].astype(np.float32))
    kappa, S = torch.from_numpy(k_h).to(dev), torch.from_numpy(s_h).to(dev)
    ib = None if Ib is None else torch.from_numpy(Ib).to(dev)
    f = torch.empty(6 * n, dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    tuning = ctx.autotune(kappa, S, ib)
    for _ in range(3):
        ctx.closure(kappa, S, ib, f)
    ctx.set_timing(True)
    stream = torch.cuda.current_stream(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    phase = []
    for i in range(steps):
        flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        ctx.closure(kappa, S, ib, f)
        ev[i][1].record(stream)
        phase.append(ctx.last_timing())
    torch.cuda.synchronize(dev)
    ctx.set_timing(False)
    ms = statistics.median(a.elapsed_time(b) for a, b in ev)
    cell_segs, face_segs = ctx.work_counts()
    cell_ms = statistics.median(ph[1] for ph in phase)
    peak = MUFU_PER_CLK_PER_SM * N_SM * float(measured_peaks().get("sm_max_mhz", 2070.0)) * 1e6 / 1e9
    achieved = cell_segs / (cell_ms * 1e-3) / 1e9
    kp, sp = torch.from_numpy(k_h).pin_memory(), torch.from_numpy(s_h).pin_memory()
    ibp = None if Ib is None else torch.from_numpy(Ib).pin_memory()
    fp = torch.empty(6 * n, dtype=torch.float32).pin_memory()
    ctx.closure(kp, sp, ibp, fp)
    t0 = time.perf_counter()
    for _ in range(3):
        ctx.closure(kp, sp, ibp, fp)
    e2e_s = (time.perf_counter() - t0) / 3
    out = {"workload": name, "value": float(n) * N / (ms * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms,
           "steps": steps, "closures_per_s": 1e3 / ms,
           "tuning": {"face_group": tuning[0], "dir_tile": tuning[1]},
           "phases_ms": {"face_pass": statistics.median(ph[0] for ph in phase), "cell_pass": cell_ms},
           "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "G exp/s",
                        "frac": achieved / peak, "traffic": None,
                        "kernel": "cell_pair_kernel<2,16> (FP32 cell pass on mirrored ray pairs)",
                        "algorithmic": f"{cell_segs} cell-ray segments (one exp each) per launch"},
           "e2e": {"value": float(n) * N / e2e_s / 1e9, "unit": UNIT, "ms_per_step": 1e3 * e2e_s,
                   "h2d_bytes_per_step": 2 * n * 4 + (0 if Ib is None else Ib.nbytes),
                   "d2h_bytes_per_step": 6 * n * 4}}
    del ctx, f, flush
    torch.cuda.empty_cache()
    if cpu:
        cores = len(os.sched_getaffinity(0))
        v, dt, used, sample = oracle_sample(p, dirs, min(N, 2 * cores), Ib, grid_text)
        out["cpu_baseline"] = {"value": v / 1e9, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample,
                               "seconds": dt}
    return out


def conv_flops_per_cell():
    """Multiply-adds x 2 of the four convolutions as stored (padded channels:
    16 -> 32 -> 32 -> 32 -> 16)."""
    return 2 * 27 * (16 * 32 + 32 * 32 + 32 * 32 + 32 * 16)


def batch_measurement(local_rank, reps: int = 20):
    """64 ragged grids (edges 32..96, block edges 8 and 16, nside 2 and 4,
    lognormal fields; synth.batched_problems) as one batched closure (one
    CUDA graph, tiles autotuned per grid shape) against the same grids'
    closures launched one after another, inputs resident in HBM."""
    import numpy as np
    import torch

    from paper_2202_08778_gb300 import synth, vet

    dev = torch.device("cuda", local_rank)
    probs = synth.batched_problems(n_grids=64, seed0=100)
    k = [torch.from_numpy(p["kappa"].astype(np.float32)).to(dev) for p in probs]
    s = [torch.from_numpy(p["S"].astype(np.float32)).to(dev) for p in probs]
    f = [torch.empty(6 * p["kappa"].size, dtype=torch.float32, device=dev) for p in probs]
    b = vet.Batch([(p["kappa"].shape, p["B"], p["h"], p["nside"], p["q"]) for p in probs], device=local_rank)
    b.autotune(k, s)
    updates = sum(p["kappa"].size * 12 * p["nside"] ** 2 for p in probs)

    def timed(fn, n):
        for _ in range(3):
            fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(n):
            fn()
        e1.record()
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / n

    def sequential():
        for i, c in enumerate(b.members):
            c.closure(k[i], s[i], None, f[i])

    t_batch = timed(lambda: b.closure(k, s, None, f), reps)
    b.sync()
    t_seq = timed(sequential, max(3, reps // 4))
    return {"workload": "64 ragged lognormal grids (synth.batched_problems, seed0 100)", "grids": len(probs),
            "ms": t_batch, "value": updates / (t_batch * 1e-3) / 1e9, "unit": UNIT, "ms_sequential": t_seq,
            "speedup_vs_sequential": t_seq / t_batch}


def hlle_measurement(ctx, kappa, S, flush, reps: int = 20):
    """The HLLE face wavespeed with the optical-depth correction (paper Sec.
    2.2.3; vet_hlle_wavespeed) from this workload's f and kappa (as rho
    kappa_R), repeated 8 times along z (16.8M cells), x-normal faces; against
    the HBM copy bandwidth: per face f_aa and kappa read (4 + 4 bytes, each
    cell once from DRAM) and the speed written (4 bytes), L2 flushed before
    every timed launch."""
    import torch

    from paper_2202_08778_gb300 import vet

    n0 = kappa.numel()
    nz, ny, nx = 128, 128, 128
    f0 = torch.empty(6 * n0, dtype=torch.float32, device=kappa.device)
    ctx.closure(kappa, S, None, f0)
    f = f0.view(6, n0).repeat(1, 8).reshape(-1)
    k = kappa.reshape(-1).repeat(8)
    shape = (8 * nz, ny, nx)
    nface = 8 * nz * ny * (nx + 1)
    C = torch.empty(nface, dtype=torch.float32, device=kappa.device)
    ms = []
    for i in range(reps + 3):
        flush.fill_(i & 255)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        vet.hlle_wavespeed(shape, 1.0 / 128, f, k, C, 0)
        b.record()
        torch.cuda.synchronize()
        if i >= 3:
            ms.append(a.elapsed_time(b))
    t = statistics.median(ms)
    nbytes = 8.0 * (8 * n0) + 4.0 * nface
    gbs = nbytes / (t * 1e-3) / 1e9
    peak = float(measured_peaks().get("hbm_gbs", 6800.0))
    return {"kernel": "hlle_kernel (vet_hlle_wavespeed, x-normal faces)", "faces": nface,
            "input": "the workload's f and kappa (as rho kappa_R) repeated 8 times along z", "ms": t,
            "bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
            "algorithmic": "8 bytes per cell read (f_xx, kappa), 4 bytes per face written",
            "G_faces_per_s": nface / (t * 1e-3) / 1e9}


def local_closure_measurement(ctx, kappa, S, flush, reps: int = 20):
    """The M1 local closure (paper Sec. 4.1; vet_local_closure) on the
    moments of this workload, against the HBM copy bandwidth: 16 bytes read
    and 24 written per cell, L2 flushed before every timed launch."""
    import torch

    from paper_2202_08778_gb300 import vet

    n0 = kappa.numel()
    M0 = torch.empty(10 * n0, dtype=torch.float32, device=kappa.device)
    f = torch.empty(6 * n0, dtype=torch.float32, device=kappa.device)
    ctx.closure(kappa, S, None, f, M0)
    # the workload's moments repeated 8 times (16.8M cells, 671 MB moved per
    # launch), so that the launch's ramp is small against its traffic
    M = M0.view(10, n0).repeat(1, 8).reshape(-1)
    n = 8 * n0
    T = torch.empty(6 * n, dtype=torch.float32, device=kappa.device)
    ms = []
    for i in range(reps + 3):
        flush.fill_(i & 255)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        vet.local_closure(vet.VET_CLOSURE_M1, M, T, n)
        b.record()
        torch.cuda.synchronize()
        if i >= 3:
            ms.append(a.elapsed_time(b))
    t = statistics.median(ms)
    gbs = 40.0 * n / (t * 1e-3) / 1e9
    peak = float(measured_peaks().get("hbm_gbs", 6800.0))
    # how far the local closure is from the ray-traced one on this field
    d = (T.view(6, n)[:, :n0] - f.view(6, n0)).abs().amax(dim=0)  # the first copy's cells
    vs_vet = {"mean": float(d.mean()), "p99": float(d.quantile(0.99)) if n0 <= (1 << 24) else None,
              "max": float(d.max())}
    return {"kernel": "m1_kernel (vet_local_closure, VET_CLOSURE_M1)", "cells": n,
            "input": "the workload's moments (vet_closure) repeated 8 times", "ms": t,
            "bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
            "algorithmic": "40 bytes per cell (E, F read; 6 components written)",
            "max_abs_dT_vs_vet": vs_vet}


def point_source_measurement(kappa, shape, h, flush, reps: int = 10):
    """The point-source deposition (paper Sec. 2.2.6; vet_point_source) of
    a source at the centre of this workload's grid, opacity = its kappa.
    Work unit: a cell a ray crosses, counted as the planes between the
    source and the cell centre plus one."""
    import numpy as np
    import torch

    from paper_2202_08778_gb300 import vet

    nz, ny, nx = shape
    n = nz * ny * nx
    xs = (0.5 * nx * h, 0.5 * ny * h, 0.5 * nz * h)
    E = torch.empty(n, dtype=torch.float32, device=kappa.device)
    p = torch.empty(3 * n, dtype=torch.float32, device=kappa.device)
    ms = []
    for r in range(reps + 3):
        flush.fill_(r & 255)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        vet.point_source(shape, h, xs, 1.0, kappa, E, p)
        b.record()
        torch.cuda.synchronize()
        if r >= 3:
            ms.append(a.elapsed_time(b))
    t = statistics.median(ms)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cross = float((np.abs(i - nx // 2 + (i < nx // 2)) + np.abs(j - ny // 2 + (j < ny // 2))
                   + np.abs(k - nz // 2 + (k < nz // 2)) + 1).sum())
    return {"kernel": "point_kernel (vet_point_source)", "workload": "source at the grid centre, kappa of the workload",
            "cells": n, "ms": t, "cell_crossings": cross, "G_crossings_per_s": cross / (t * 1e-3) / 1e9,
            "rate": n / (t * 1e-3) / 1e9, "rate_unit": "G cells/s"}


def reuse_measurement(ctx, flush, steps: int = 12, cells_per_step: float = 0.01, reps: int = 10):
    """Reuse of f across time steps (paper Sec. 4.2; vet_field_change and
    vet.ClosureReuse) on the workload's lognormal fields carried 0.01 cells
    per step: per tolerance the steps that recompute, the time per step
    (gate, 12-byte read-back and the closures it runs) and the largest
    difference from a fresh f; and the gate kernel against the HBM copy
    bandwidth on the fields repeated 8 times along z (L2 flushed before
    every timed launch; 16 bytes read per cell, 24 with the snapshot)."""
    import torch

    from paper_2202_08778_gb300 import synth, vet

    p, seq = synth.lognormal_sequence(n=128, B=16, nside=4, seed=2, steps=steps, cells_per_step=cells_per_step)
    dev = flush.device
    fields = [(torch.from_numpy(k.ravel()).to(dev), torch.from_numpy(s.ravel()).to(dev)) for k, s in seq]
    n = ctx.ncell
    fresh = []
    for k, s in fields:
        f = torch.empty(6 * n, dtype=torch.float32, device=dev)
        ctx.closure(k, s, None, f)
        fresh.append(f)
    torch.cuda.synchronize(dev)
    runs = []
    for tol in (0.0, 0.02, 0.05, 0.1):
        run = vet.ClosureReuse(ctx, tol_tau=tol, tol_S=tol, max_age=8)
        err = []
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for t, (k, s) in enumerate(fields):
            f, _ = run.step(k, s)
        torch.cuda.synchronize(dev)
        dt = (time.perf_counter() - t0) / steps
        run2 = vet.ClosureReuse(ctx, tol_tau=tol, tol_S=tol, max_age=8)
        flags = []
        for t, (k, s) in enumerate(fields):  # same decisions, errors taken outside the timed loop
            f, redo = run2.step(k, s)
            flags.append(bool(redo))
            err.append(float((f - fresh[t]).abs().max()))
        runs.append({"tol": tol, "recomputed_steps": [i for i, r in enumerate(flags) if r],
                     "ms_per_step": 1e3 * dt, "cell_angle_per_s_G": n * ctx.N / dt / 1e9,
                     "max_abs_df": max(err), "max_abs_df_per_step": err})
    # the gate kernel alone, on 8 copies of the fields stacked along z
    k0, s0 = fields[0]
    k1, s1 = fields[1]
    nz, ny, nx = ctx.shape
    big = [x.repeat(8) for x in (k1, s1, k0, s0)]
    nb = 8 * n // ctx.block ** 3
    out = torch.empty(3 + 3 * nb, dtype=torch.float32, device=dev)
    res = {}
    for snap in (False, True):
        ms = []
        for r in range(reps + 3):
            flush.fill_(r & 255)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            vet.field_change((8 * nz, ny, nx), ctx.block, ctx.h, *big, out, snap)
            b.record()
            torch.cuda.synchronize(dev)
            if r >= 3:
                ms.append(a.elapsed_time(b))
        res[snap] = statistics.median(ms)
    peak = float(measured_peaks().get("hbm_gbs", 6800.0))
    gbs = 16.0 * 8 * n / (res[False] * 1e-3) / 1e9
    gbs_snap = 24.0 * 8 * n / (res[True] * 1e-3) / 1e9
    ms1 = []
    kr, sr = k0.clone(), s0.clone()
    out1 = torch.empty(3 + 3 * (n // ctx.block ** 3), dtype=torch.float32, device=dev)
    for r in range(reps + 3):
        flush.fill_(r & 255)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        vet.field_change(ctx.shape, ctx.block, ctx.h, k1, s1, kr, sr, out1, False)
        b.record()
        torch.cuda.synchronize(dev)
        if r >= 3:
            ms1.append(a.elapsed_time(b))
    return {"workload": f"lognormal128 fields carried {cells_per_step} cells per step, {steps} steps",
            "runs": runs, "max_age": 8,
            "gate": {"kernel": "gate_kernel<true> (vet_field_change)", "cells": 8 * n,
                     "input": "two steps' fields repeated 8 times along z", "ms": res[False],
                     "bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                     "algorithmic": "16 bytes read per cell (kappa, S, kappa_ref, S_ref)",
                     "snapshot": {"ms": res[True], "achieved": gbs_snap, "frac": gbs_snap / peak,
                                  "algorithmic": "16 bytes read and 8 written per cell"},
                     "us_at_128cubed": 1e3 * statistics.median(ms1)}}


def learned_measurement(local_rank):
    """The learned closure at 256^3 in 16^3 blocks with 192 directions (the
    lognormal generator, seed 3) against the plain closure on the same GPU.
    The network is trained here, on 64^3 snapshots of the same generator
    labelled by the exact closure (a bounded sample of the specified 2000)."""
    import numpy as np
    import torch

    from paper_2202_08778_gb300 import learned, synth, vet

    dev = torch.device("cuda", local_rank)
    nt, B, ns = 64, 16, 4
    ntrain, steps, batch = 64, 1500, 4
    t0 = time.perf_counter()
    ctx_t = vet.Context((nt,) * 3, B, 1.0 / nt, ns, synth.rotation_quaternion(10000), device=local_rank)
    data = learned.snapshots(ctx_t, range(10000, 10000 + ntrain), nt, B, ns)
    t_data = time.perf_counter() - t0
    model = vet.Model(device=local_rank)
    model.set_params(learned.init_params(32, seed=0))
    t0 = time.perf_counter()
    losses = learned.train(model, data, (nt,) * 3, B, 1.0 / nt, steps, batch=batch)
    torch.cuda.synchronize(dev)
    t_train = time.perf_counter() - t0
    del data, ctx_t

    n = 256
    p = synth.lognormal_problem(n=n, B=B, nside=ns, seed=3)
    ctx = vet.Context(p["kappa"].shape, B, p["h"], ns, p["q"], device=local_rank)
    kappa = torch.from_numpy(np.ascontiguousarray(p["kappa"].astype(np.float32))).to(dev)
    S = torch.from_numpy(np.ascontiguousarray(p["S"].astype(np.float32))).to(dev)
    N = n ** 3
    nblk = N // B ** 3
    f_plain = torch.empty(6 * N, device=dev)
    M = torch.empty(10 * N, device=dev)
    ctx.autotune(kappa, S)
    ctx.closure(kappa, S, None, f_plain, M)
    E = M[:N].clone()
    del M
    ctx.set_timing(True)
    plain = []
    for _ in range(5):  # the working set (3 GB of faces) is far larger than L2
        ctx.closure(kappa, S, None, f_plain)
        plain.append(ctx.last_timing()[3])
    ctx.set_timing(False)
    plain_ms = statistics.median(plain)

    f = torch.empty(6 * N, device=dev)

    def run(thr):
        model.closure(ctx, kappa, S, E, f, threshold=thr)
        ts = []
        nfb = 0
        for _ in range(3):
            nfb = model.closure(ctx, kappa, S, E, f, threshold=thr)
            ts.append(model.last_timing())
        ctx.sync()
        return nfb, [statistics.median(t[i] for t in ts) for i in range(4)]

    def err_stats(fg):
        e = (fg - f_plain).abs().view(6, -1).amax(0)
        q = torch.quantile(e[::97].double(), torch.tensor([0.5, 0.99], dtype=torch.float64, device=dev))
        return {"mean": float(e.double().mean()), "p50": float(q[0]), "p99": float(q[1]), "max": float(e.max())}

    nfb_inf, t_inf = run(float("inf"))
    net_err = err_stats(f)
    thr = 1e-2
    nfb, t_thr = run(thr)
    fb_err = float((f - f_plain).abs().max())
    iso = torch.zeros_like(f).view(6, -1)
    iso[:3] = 1.0 / 3.0
    edd = (iso - f_plain.view(6, -1)).abs().amax(0)
    tflops = conv_flops_per_cell() * N / (t_inf[3] * 1e-3) / 1e12
    peak = float(measured_peaks().get("bf16_tflops", 1900.0))
    return {
        "workload": "lognormal256_B16_nside4 (seed 3)", "plain_closure_ms": plain_ms,
        "threshold": thr, "fallback_blocks": nfb, "blocks": nblk, "ms": t_thr[2],
        "ms_network": t_thr[0], "ms_fallback": t_thr[1], "speedup_vs_plain": plain_ms / t_thr[2],
        "max_abs_df_vs_plain": fb_err,
        "network_only": {"ms": t_inf[2], "speedup_vs_plain": plain_ms / t_inf[2], "abs_df_vs_plain": net_err},
        "eddington_I_over_3": {"mean": float(edd.double().mean()), "max": float(edd.max())},
        "conv_roofline": {"bound": "tensor", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                          "frac": tflops / peak, "kernel": "conv3d_tc_kernel (4 layers, tcgen05 BF16, FP32 accumulators in TMEM)",
                          "algorithmic": f"{conv_flops_per_cell()} FLOP per cell (padded channels) x {N} cells"},
        "train": {"snapshots": ntrain, "shape": [nt] * 3, "steps": steps, "batch": batch,
                  "seconds": t_train, "data_seconds": t_data, "final_loss": losses[-1]},
    }


def run_reference(args, rank, world):
    """The oracle as the reference arm (host cores, rank 0 only)."""
    if rank != 0:
        return
    import numpy as np

    import oracle

    p, cfg = workload()
    oracle.build()
    dirs = oracle.healpix(p["nside"], p["q"])
    cores = len(os.sched_getaffinity(0))
    nsub = min(dirs.shape[0], max(4, cores))
    for _ in range(args.warmup):
        oracle_sample(p, dirs, nsub)
    ts = []
    for _ in range(args.steps):
        v, dt, used, sample = oracle_sample(p, dirs, nsub)
        ts.append(dt)
    upd = p["kappa"].size * nsub
    value = upd * len(ts) / sum(ts) / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(ts) / len(ts),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_2202_08778_gb300 import vet

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    p, cfg = workload()
    n = p["kappa"].size
    ctx = vet.Context(p["kappa"].shape, p["B"], p["h"], p["nside"], p["q"], device=local_rank)
    N = ctx.N
    k_h = np.ascontiguousarray(p["kappa"].astype(np.float32))
    s_h = np.ascontiguousarray(p["S"].astype(np.float32))
    kappa = torch.from_numpy(k_h).to(dev)
    S = torch.from_numpy(s_h).to(dev)
    f = torch.empty(6 * n, dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    cell_segs, face_segs = ctx.work_counts()
    launches = ctx.launches_per_closure()

    if args.tuning:  # fixed tiles (profiling: the autotuner's timings are not meaningful under ncu)
        ctx.set_tuning(*args.tuning)
        tuning = ctx.tuning()
    else:
        tuning = ctx.autotune(kappa, S)  # the library's own tile choice, before timing
    cfg["tuning"] = {"face_group": tuning[0], "dir_tile": tuning[1], "autotuned": not args.tuning}
    for _ in range(args.warmup):
        ctx.closure(kappa, S, None, f)
    ctx.set_timing(True)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    phase = []
    with ClockSampler(local_rank) as clk:
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            ctx.closure(kappa, S, None, f)
            ev[i][1].record(stream)
            phase.append(ctx.last_timing())
        torch.cuda.synchronize(dev)
    ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = slowest_rank_ms(sum(ms), world, dev)
    ctx.set_timing(False)
    ms_step = total_ms / args.steps
    value = whole_job_rate(float(n) * N * args.steps, world, total_ms) / 1e9

    # end to end through the C ABI with host buffers (pinned), copies inside
    kp = torch.from_numpy(k_h).pin_memory()
    sp = torch.from_numpy(s_h).pin_memory()
    fp = torch.empty(6 * n, dtype=torch.float32).pin_memory()
    ctx.closure(kp, sp, None, fp)
    e2e_steps = max(3, min(args.steps, 20))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.closure(kp, sp, None, fp)  # stages H2D, computes, D2H, synchronises
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e = {"value": float(n) * N / e2e_s / 1e9, "unit": UNIT, "h2d_bytes_per_step": 2 * n * 4,
           "d2h_bytes_per_step": 6 * n * 4, "ms_per_step": 1e3 * e2e_s}

    local = local_closure_measurement(ctx, kappa, S, flush) if rank == 0 and world == 1 else None
    hlle = hlle_measurement(ctx, kappa, S, flush) if rank == 0 and world == 1 else None
    point = (point_source_measurement(kappa, p["kappa"].shape, p["h"], flush)
             if rank == 0 and world == 1 else None)

    # roofline of the dominant kernel (the cell pass), from the live events
    cell_ms = statistics.median(ph[1] for ph in phase)
    face_ms = statistics.median(ph[0] for ph in phase)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak = MUFU_PER_CLK_PER_SM * N_SM * sm_max * 1e6 / 1e9  # G exp/s
    achieved = cell_segs / (cell_ms * 1e-3) / 1e9
    traffic = measured_traffic()
    try:  # the unit count behind the peak, measured on this GPU
        from paper_2202_08778_gb300 import peaks as _peaks

        units = _peaks.measure()
    except Exception as exc:  # noqa: BLE001 - reported, not fatal
        units = {"error": str(exc)[:200]}
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "G exp/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": "cell_pair_kernel<2,16> (FP32 cell pass on mirrored ray pairs)",
                "peak_basis": f"MUFU ex2: {MUFU_PER_CLK_PER_SM}/clk/SM x {N_SM} SMs x {sm_max:.0f} MHz",
                "algorithmic": f"{cell_segs} cell-ray segments (one exp each) per launch",
                "measured_units_per_clk_per_sm": units}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
            "closures_per_s": 1e3 / ms_step * world,
            "phases_ms": {"face_pass": face_ms, "cell_pass": cell_ms,
                          "closing": statistics.median(ph[2] for ph in phase)},
            "work": {"cell_segments": cell_segs, "face_segments": face_segs,
                     "segments_per_cell_angle": (cell_segs + face_segs) / (n * N)},
            "roofline": roofline, "e2e": e2e, "gpu_launches": launches * args.steps}
    if local is not None:
        line["local_closure_m1"] = local
    if hlle is not None:
        line["hlle_wavespeed"] = hlle
    if point is not None:
        line["point_source"] = point
    clocks = clk.summary()
    if clocks is not None:
        line["clocks"] = clocks

    if rank == 0 and world == 1 and not args.no_reuse:
        line["reuse"] = reuse_measurement(ctx, flush)

    if rank == 0 and world == 1 and not args.no_large:
        line["workloads"] = {kind: workload_measurement(local_rank, kind, cpu=not args.no_cpu_baseline)
                             for kind in ("shadow", "lognormal256")}

    if rank == 0 and world == 1 and not args.no_batch:
        line["batch"] = batch_measurement(local_rank)

    if rank == 0 and world == 1 and not args.no_learned:
        line["learned"] = learned_measurement(local_rank)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = len(os.sched_getaffinity(0))
        nsub = min(N, 2 * cores)
        v, dt, used, sample = oracle_sample(p, ctx.directions(), nsub)
        line["cpu_baseline"] = {"value": v / 1e9, "unit": UNIT, "cores": used, "kind": "oracle",
                                "sample": sample, "seconds": dt}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-closure measurement")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-grid batched-closure measurement")
    ap.add_argument("--no-reuse", action="store_true", help="skip the measurement of reusing f across time steps")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the 256x128x128 shadow and 256^3 lognormal workloads")
    ap.add_argument("--tuning", type=lambda v: tuple(int(x) for x in v.split(",")), default=None,
                    metavar="FG,DT", help="fixed face-pass direction group and cell-pass direction tile "
                    "instead of autotuning")
    args = ap.parse_args()
    if args.tuning is not None and len(args.tuning) != 2:
        ap.error("--tuning takes two integers: FG,DT")
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch

        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch

            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
