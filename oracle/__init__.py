"""FP64 CPU oracle for the direct-summation Hermite hot path of arXiv:0902.4463.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product package
never imports it, and it never imports the product package.

The arithmetic lives in ``oracle.c`` (plain C, double precision, one OpenMP loop
over i-particles); ``oracle.py`` only marshals numpy arrays through ctypes.

Parity status: every function is pinned by ``tests/test_oracle_pins.py``
(closed forms, finite differences, conservation laws, constructed cases),
except the choice of the Aarseth step at the end rather than the start of a
step inside ``orc_hermite_run``, which no closed form distinguishes.
"""
from .oracle import (  # noqa: F401
    Oracle,
    aarseth_dt,
    block_dt,
    build,
    compile_source,
    default,
    energy,
    force,
    hermite_correct,
    hermite_run,
    lib_path,
    neighbours,
    predict,
)
