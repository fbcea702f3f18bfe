"""The C ABI library builds, loads without a GPU and exports exactly the
entry points include/*.h declares (no compute call is made here)."""
import ctypes
import glob
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?(?:\w+\s+)*?\w+\s*\**\s*(vet_\w+)\s*\(", src, flags=re.M))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("vet_trace", "vet_moments", "vet_closure", "vet_create", "vet_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2202_08778_gb300 import build, vet

    path = build.build()
    lib = ctypes.CDLL(path)
    for n in _declared():
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert exported == _declared()
    assert set(vet.EXPORTS) == _declared()


def test_create_without_gpu_fails_cleanly():
    import torch

    if torch.cuda.is_available():
        return
    from paper_2202_08778_gb300 import vet

    try:
        vet.Context((8, 8, 8), 4, 0.1, 1)
    except vet.VetError as e:
        assert e.status == vet.VET_ECUDA
    else:  # pragma: no cover
        raise AssertionError("vet_create succeeded without a GPU")


def test_binding_declares_argument_types_of_every_entry_point():
    """Without argtypes ctypes passes Python ints as 32-bit C ints, which
    truncates 64-bit device pointers."""
    from paper_2202_08778_gb300 import vet

    lib = vet.load()
    for n in vet.EXPORTS:
        assert getattr(lib, n).argtypes is not None, n
