"""Build libvet (the CUDA library behind include/vet.h) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into
paper_2202_08778_gb300/_build/libvet.so (static CUDA runtime, only the C ABI
exported).  No cmake; a minute or less on either host architecture.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libvet.so")
SOURCES = ["vet_host.cu", "vet_kernels.cu", "vet_noalloc.cu", "vet_cnn.cu", "vet_cnn_tc.cu", "vet_learned.cu",
           "vet_local.cu", "vet_point.cu", "vet_reuse.cu", "vet_hlle.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: libvet cannot be built")


def _inputs():
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    files.append(os.path.join(INCLUDE, "vet.h"))
    return files


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _inputs())


def build(force: bool = False, verbose: bool = False, extra_flags=None) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()
    extra = list(extra_flags or [])

    def compile_one(src):
        obj = os.path.join(OUT_DIR, os.path.splitext(src)[0] + ".o")
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fPIC"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


PEAKS = os.path.join(OUT_DIR, "vet_peaks")


def build_peaks(force: bool = False) -> str:
    """Compile the unit-rate microbenchmark (csrc/peaks.cu) into an
    executable next to libvet."""
    src = os.path.join(CSRC, "peaks.cu")
    if not force and os.path.exists(PEAKS) and os.path.getmtime(PEAKS) >= os.path.getmtime(src):
        return PEAKS
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = PEAKS + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc(), *ARCH, "-O3", "-std=c++17", src, "-o", tmp], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on peaks.cu:\n{r.stderr}")
    os.replace(tmp, PEAKS)
    return PEAKS


if __name__ == "__main__":
    print(build(force=True, verbose=True))
