"""Run a Plummer model with the library's Hermite block-time-step driver.

    python -m paper_0902_4463_gb300.hermite_run --n 32768 --seed 2 --eps2 1e-5 \
        --eta 0.01 --t-end 1 --prec ds

The force path runs on the GPU through the C ABI (Sect. 2: the library
predicts the j-particles and computes forces, the host C++ driver predicts
the i-particles, corrects them and picks block time steps).  Energies are
evaluated with one all-FP64 force sweep through the same library, so that the
drift measures the integration, not the energy evaluation.

Prints one JSON line: wall time, block steps, sum of block sizes, mean block
size, interactions/s and 60-flop Gflop/s over the whole run, the block-size
histogram (log2 bins), dE/E = (E1 - E0)/E0 (Sect. 3.2) and, with --h2, the
neighbour lists read back (Sect. 4: count, entries, overflows).
"""
import argparse
import json
import math
import sys
import time

import numpy as np

from . import build as _build
from . import g6gb as g6
from . import ics

PREC = {"ds": g6.G6X_PREC_DS, "fp64": g6.G6X_PREC_FP64, "ds_x64": g6.G6X_PREC_DS_X64,
        "ds_dssub": g6.G6X_PREC_DS_DSSUB}


def energy_fp64(cid, sim, mode):
    g6.g6x_set_precision(cid, g6.G6X_PREC_FP64)
    try:
        ek, ep = sim.energy()
    finally:
        g6.g6x_set_precision(cid, mode)
    return ek + ep


def run(n, seed, eps2, eta, t_end, prec="ds", binaries=0.0, dt_max=2.0 ** -4, cid=0,
        tune=None, h2=0.0, noise=0.0, maxnb=0):
    """Integrate and return the result dict (the context is opened and closed
    here)."""
    _build.build()
    if binaries > 0:
        m, x, v, _ = ics.plummer_with_binaries(n, seed, fbin=binaries)
    else:
        m, x, v = ics.plummer(n, seed)
    mode = PREC[prec]
    g6.g6x_open_ex(cid, n, n)
    try:
        g6.g6x_set_precision(cid, mode)
        if tune:
            g6.g6x_load_tuning(tune)
        if maxnb > 0:
            g6.g6x_set_max_neighbours(cid, maxnb)
        sim = g6.G6HSim(cid, m, x, v, eps2, eta, dt_max=dt_max)
        if h2 > 0:
            sim.set_neighbour_radius(h2)
        if noise > 0:
            sim.set_force_noise(noise)
        e0 = energy_fp64(cid, sim, mode)
        t0 = time.perf_counter()
        sim.run(t_end)
        wall = time.perf_counter() - t0
        st = sim.stats()
        prof = sim.profile()
        nbs = sim.neighbour_stats()
        e1 = energy_fp64(cid, sim, mode)
        state = sim.state()
        sim.close()
    finally:
        g6.g6_close(cid)
    inter = float(st["nactive"]) * n
    hist = {int(2 ** b): int(c) for b, c in enumerate(st["hist"]) if c}
    return dict(n=n, seed=seed, eps2=eps2, eta=eta, t_end=t_end, prec=prec,
                binaries=binaries, wall_s=wall, nblocks=int(st["nblocks"]),
                nactive=int(st["nactive"]), mean_block=st["nactive"] / max(1, st["nblocks"]),
                interactions_per_s=inter / wall, gflops_60=60.0 * inter / wall / 1e9,
                dE_over_E=(e1 - e0) / e0, E0=e0, E1=e1, block_hist_log2=hist,
                profile=prof, h2=h2, force_noise=noise, neighbour_lists=nbs,
                max_neighbours=maxnb or g6.G6_MAXNB,
                synchronised=bool(np.all(state["t"] == t_end)))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=32768)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--eps2", type=float, default=1e-5)
    ap.add_argument("--eta", type=float, default=0.01)
    ap.add_argument("--t-end", type=float, default=1.0)
    ap.add_argument("--prec", default="ds", choices=sorted(PREC))
    ap.add_argument("--binaries", type=float, default=0.0,
                    help="fraction of stars in equal-mass binaries")
    ap.add_argument("--tune", default=None, help="autotuner table to load")
    ap.add_argument("--h2", type=float, default=0.0,
                    help="neighbour-list radius^2 requested every block step (0: none)")
    ap.add_argument("--noise", type=float, default=0.0,
                    help="relative force error the time-step choice allows for (0: none)")
    ap.add_argument("--maxnb", type=int, default=0,
                    help="neighbour-list length (0: the default, 256)")
    a = ap.parse_args(argv)
    r = run(a.n, a.seed, a.eps2, a.eta, a.t_end, a.prec, a.binaries, tune=a.tune, h2=a.h2,
            noise=a.noise, maxnb=a.maxnb)
    print(json.dumps(r))
    return 0


if __name__ == "__main__":
    sys.exit(main())
