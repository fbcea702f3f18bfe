"""FP64 CPU oracle for the VET closure (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does.
"""
from .oracle import (  # noqa: F401
    build,
    healpix,
    trace,
    moments,
    closure,
    count_segments,
    vet_closure,
)
