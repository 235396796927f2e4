"""Per-call cost of small block steps through the GRAPE calling sequence.

    python -m paper_0902_4463_gb300.block_latency --n 32768 --reps 300 [--tune]

Builds the library, compiles the plain C program `block_latency.c` against it
(gcc, into the package's `_build/`), and runs it: for m = 1 .. 4096 active
particles against n j-particles, the host wall time of each call of one block
step (j-update, block time, firsthalf, lasthalf) and the device time of each
phase (CUDA events), one JSON line per m.  The calls are timed from C so that
no binding overhead enters the host numbers.
"""
import argparse
import os
import subprocess
import sys

from . import build as _build


def compile_tool():
    _build.build()
    src = os.path.join(_build.HERE, "block_latency.c")
    os.makedirs(_build.OBJDIR, exist_ok=True)
    exe = os.path.join(_build.OBJDIR, "block_latency")
    newest = max(os.path.getmtime(src), os.path.getmtime(_build.LIB),
                 os.path.getmtime(os.path.join(_build.INCLUDE, "g6gb.h")))
    if not os.path.exists(exe) or os.path.getmtime(exe) < newest:
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-I", _build.INCLUDE, src,
                               "-L", _build.HERE, "-lg6gb", "-Wl,-rpath," + _build.HERE,
                               "-o", exe])
    return exe


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=32768)
    ap.add_argument("--reps", type=int, default=300)
    ap.add_argument("--tune", action="store_true", help="run the autotuner at this n first")
    a = ap.parse_args(argv)
    cmd = [compile_tool(), str(a.n), str(a.reps)] + (["tune"] if a.tune else [])
    return subprocess.call(cmd)


if __name__ == "__main__":
    sys.exit(main())
