"""Oracle of the change gate for reusing the Eddington tensor across time
steps (paper Sec. 4.2, "Performance": the suggestion that f need not be
recomputed at the start of every time step).

TEST INFRASTRUCTURE: imported only by the tests and the benchmark; it shares
nothing with the product library.

The paper gives no criterion for when a stored f may be reused; the reading
taken here measures how far the closure's two cell inputs moved since the
snapshot the stored f was computed from, per block of B^3 cells and over the
grid:
  dtrans = max_c |a - b| / ((1 + a/2) (1 + b/2)),  a = kappa_c h,
                                                   b = kappa_ref_c h
           an upper bound on the change |e^{-a} - e^{-b}| of the cell's
           transmission (from e^t >= (1 + t/2)^2, so e^{-t} <= (1 + t/2)^-2,
           integrated from min(a, b) to max(a, b)); a cell's outgoing
           intensity I e^{-tau} + S (1 - e^{-tau}) (the solution of Eq. 14
           across it) moves by (S - I) times that change, so an optically
           thick cell whose opacity changes does not count, while for thin
           cells dtrans ~ |a - b|;
  dS     = max_c |S_c - S_ref_c|            (largest change of the source)
  Sref   = max_c |S_ref_c|                  (scale of the source)
The gate's decision compares dtrans with an absolute tolerance and dS with a
tolerance relative to Sref (f = P / E does not change when S is scaled).

Arithmetic: float32, as the product computes it, so both sides take the
decision on the same numbers: a, b, the difference, each factor
1 + t/2 (t/2 is exact), their product and the quotient are one IEEE
rounding each, and a maximum is exact.  A NaN anywhere counts as +inf (a
non-finite input always forces a recompute).

Layout: fields [nz][ny][nx] float32; blocks of B^3 cells numbered x-fastest,
b = (bk * nby + bj) * nbx + bi.  Result [3 + 3 * nblocks] float32: the grid's
(dtrans, dS, Sref), then each block's triple.
"""
from __future__ import annotations

import numpy as np


def _block_max(a: np.ndarray, B: int) -> np.ndarray:
    nz, ny, nx = a.shape
    v = a.reshape(nz // B, B, ny // B, B, nx // B, B)
    return v.max(axis=(1, 3, 5)).reshape(-1)  # blocks x-fastest


def change(kappa, S, kappa_ref, S_ref, h: float, B: int) -> np.ndarray:
    """(dtrans, dS, Sref) of the grid and of every block, float32."""
    k, s = np.asarray(kappa, np.float32), np.asarray(S, np.float32)
    kr, sr = np.asarray(kappa_ref, np.float32), np.asarray(S_ref, np.float32)
    nz, ny, nx = k.shape
    if nz % B or ny % B or nx % B:
        raise ValueError("the block edge must divide every extent")
    h32, half, one = np.float32(h), np.float32(0.5), np.float32(1.0)
    with np.errstate(invalid="ignore", over="ignore", divide="ignore"):
        a = k * h32
        b = kr * h32
        dtau = np.abs(a - b) / ((one + half * a) * (one + half * b))
        dS = np.abs(s - sr)
    dtau = np.where(np.isnan(dtau), np.float32(np.inf), dtau).astype(np.float32)
    dS = np.where(np.isnan(dS), np.float32(np.inf), dS).astype(np.float32)
    sref = np.abs(sr)
    sref = np.where(np.isnan(sref), np.float32(np.inf), sref).astype(np.float32)
    per = np.stack([_block_max(dtau, B), _block_max(dS, B), _block_max(sref, B)], axis=1)
    grid = per.max(axis=0)
    return np.concatenate([grid, per.reshape(-1)]).astype(np.float32)


def recompute(triple, age: int, first: bool, tol_tau: float, tol_S: float, max_age: int) -> bool:
    """The gate's decision for one time step: recompute f on the first step,
    when the stored f is max_age steps old, or when either input moved by
    more than its tolerance (a non-finite change always does)."""
    dtau, dS, sref = (float(x) for x in triple[:3])  # dtau: the transmission bound dtrans
    if first or age >= max_age:
        return True
    if not (np.isfinite(dtau) and np.isfinite(dS)):
        return True
    return dtau > tol_tau or dS > tol_S * sref
