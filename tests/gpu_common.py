"""Helpers shared by the GPU parity tests: problem set-up on both sides and
error measures.  The inputs come from the seeded generators in
paper_2202_08778_gb300.synth; the expected values from the CPU oracle."""
from __future__ import annotations

import numpy as np

FLOOR_REL = 1e-30  # the closure's isotropic-fallback threshold, relative to max E


def rel_err(got, ref, floor_rel=FLOOR_REL):
    """max |got - ref| / max(|ref|, floor_rel * max|ref|)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.maximum(np.abs(ref), floor_rel * np.abs(ref).max() + 1e-300)
    return float((np.abs(got - ref) / den).max())


def moment_errors(M_got, M_ref, E_floor_rel=FLOOR_REL):
    """(max relative error of E, max |dF|/E and |dP|/E) over cells above the
    floor; F and P errors are measured against E of the same cell because
    their components may vanish."""
    M_got = np.asarray(M_got, dtype=np.float64).reshape(10, -1)
    M_ref = np.asarray(M_ref, dtype=np.float64).reshape(10, -1)
    E = M_ref[0]
    keep = E > E_floor_rel * E.max()
    eE = (np.abs(M_got[0] - E)[keep] / E[keep]).max()
    eFP = (np.abs(M_got[1:] - M_ref[1:]).max(0)[keep] / E[keep]).max()
    return float(eE), float(eFP)


def f_error(f_got, f_ref, M_ref, floor_rel=FLOOR_REL, margin=1e-3):
    """max |f_got - f_ref| over cells whose E is clearly above or below the
    floor (cells within a relative `margin` of it may legitimately fall on
    either side); both sides must agree on which cells are isotropic."""
    f_got = np.asarray(f_got, dtype=np.float64).reshape(6, -1)
    f_ref = np.asarray(f_ref, dtype=np.float64).reshape(6, -1)
    E = np.asarray(M_ref, dtype=np.float64).reshape(10, -1)[0]
    fl = floor_rel * E.max()
    clear = (E > fl * (1 + margin)) | (E < fl * (1 - margin))
    return float(np.abs(f_got - f_ref)[:, clear].max())
