"""Host logic of the mirrored-pair passes (vet_geometry.h), compiled with the
host C++ compiler and run without a GPU: antipodes at equal positions of
opposite octants, the cell- and node-ray mirror checks, the face passes'
node order by ray length, and the paired face-pass schedule covering the
unpaired one level by level."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2202_08778_gb300", "csrc")


def _cuda_include():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "include", "cuda_runtime.h")):
            return os.path.join(c, "include")
    return None


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = _cuda_include()
    if not cxx or not inc:
        pytest.skip("no host C++ compiler or CUDA headers")
    exe = str(tmp_path_factory.mktemp("geom") / "geometry_check")
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", inc, "-I", CSRC, os.path.join(ROOT, "tests", "host", "geometry_check.cpp"),
                    "-o", exe], check=True)
    return exe


@pytest.mark.parametrize("nb,B,nside", [((8, 8, 8), 16, 4), ((4, 2, 3), 8, 2), ((3, 3, 3), 16, 2), ((1, 1, 1), 8, 1),
                                        ((5, 2, 1), 16, 4), ((2, 2, 2), 8, 8),
                                        # block edges of the unpaired passes (templates, node order, schedule)
                                        ((3, 2, 2), 12, 2), ((2, 2, 2), 32, 2)])
def test_mirrored_pairs_and_paired_schedule(checker, nb, B, nside):
    r = subprocess.run([checker, *map(str, nb), str(B), str(nside)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr


@pytest.mark.parametrize("nside", [1, 2, 4])
def test_sets_with_zero_components_are_not_paired(checker, nside):
    r = subprocess.run([checker, "2", "2", "2", "8", str(nside), "unrotated"], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
