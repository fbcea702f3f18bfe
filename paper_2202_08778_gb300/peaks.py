"""Per-SM rates of the units the closure's kernels use, measured on the GPU
by csrc/peaks.cu (MUFU ex2, FP32 FMA, f32x2 FMA, 8- and 16-byte shared-memory
loads), per SM clock.

  python -m paper_2202_08778_gb300.peaks
"""
from __future__ import annotations

import json
import subprocess

from . import build


def measure(timeout: float = 120.0) -> dict:
    exe = build.build_peaks()
    r = subprocess.run([exe], capture_output=True, text=True, timeout=timeout)
    if r.returncode != 0:
        raise RuntimeError(f"vet_peaks failed ({r.returncode}): {r.stdout.strip()} {r.stderr.strip()}")
    return json.loads(r.stdout)


if __name__ == "__main__":
    print(json.dumps(measure()))
