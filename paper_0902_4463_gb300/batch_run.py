"""Batch workload: 256 independent Plummer clusters, N log-uniform in
[256, 16384], Salpeter masses, eps2 = (4/N)^2 (ics.cluster_batch).

    python -m paper_0902_4463_gb300.batch_run --ncl 256 --seed 1 --t-end 0.0625

Two measurements, both printed as one JSON line:

* force-only batch calls (Sect. 2: one force call per block step, here for
  every cluster at once) on seeded uneven active sets: per cluster
  ni = max(1, N >> u), u uniform in 0 .. floor(log2 N), a fifth of the
  clusters idle per call.  Timed end to end per call (host staging, launch,
  wait, results in mapped memory) for every batch kernel shape x grid
  multiplier in one CUDA-graph replay (the schedule tuning: the best is
  kept), then with that schedule as plain launches and as one launch
  sequence per cluster;
* the Hermite batch driver (every cluster its own block scheduler, one batch
  force call per batch step) to t_end with the tuned schedule, graph mode
  against per-cluster launches.

Interactions count ni x N per cluster and call; Gflop/s uses 60 flops per
interaction (Sect. 3.1).
"""
import argparse
import json
import sys
import time

import numpy as np

from . import build as _build
from . import g6gb as g6
from . import ics

FLOPS = 60.0


def _patterns(cls, seed, count):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        ni = []
        for c in cls:
            n = c["n"]
            if rng.random() < 0.2:
                ni.append(0)
                continue
            u = int(rng.integers(0, int(np.log2(n)) + 1))
            ni.append(max(1, n >> u))
        out.append(np.array(ni, dtype=np.int32))
    return out


def _make_batch(cls, variant, grid_mul):
    b = g6.G6Batch([c["n"] for c in cls], variant=variant, grid_mul=grid_mul)
    for k, c in enumerate(cls):
        b.set_j(k, c["m"], c["x"], c["v"])
        b.set_i(k, c["x"], c["v"])
    return b


def force_calls(cls, variant, grid_mul, mode, patterns, reps):
    """Mean seconds per batch call and interactions per call."""
    b = _make_batch(cls, variant, grid_mul)
    try:
        eps2 = np.array([c["eps2"] for c in cls])
        n = np.array([c["n"] for c in cls])
        t = np.zeros(len(cls))
        b.calc(t, eps2, n, mode)                 # staging, graph capture, warm-up
        for p in patterns:
            b.calc(t, eps2, p, mode)
        t0 = time.perf_counter()
        for _ in range(reps):
            for p in patterns:
                b.calc(t, eps2, p, mode)
        sec = (time.perf_counter() - t0) / (reps * len(patterns))
        inter = float(np.mean([np.dot(p.astype(np.float64), n) for p in patterns]))
        return sec, inter, b.launch_count()
    finally:
        b.close()


def driver(cls, variant, grid_mul, mode, t_end, eta):
    sim = g6.G6HBatchSim([(c["m"], c["x"], c["v"]) for c in cls],
                         [c["eps2"] for c in cls], eta, variant=variant,
                         grid_mul=grid_mul, mode=mode)
    try:
        t0 = time.perf_counter()
        sim.run(t_end)
        wall = time.perf_counter() - t0
        st = sim.stats()
        ok = bool(np.all(sim.state()["t"] == t_end))
    finally:
        sim.close()
    return dict(mode=mode, wall_s=wall, batch_steps=st["nsteps"], nactive=st["nactive"],
                interactions=st["interactions"], sec_gpu=st["sec_gpu"],
                sec_host=st["sec_host"], interactions_per_s=st["interactions"] / wall,
                gflops_60=FLOPS * st["interactions"] / wall / 1e9,
                us_per_batch_step=1e6 * wall / max(1, st["nsteps"]), synchronised=ok)


def run(ncl=256, seed=1, t_end=0.0625, eta=0.01, npat=16, reps=3, variants=None,
        grid_muls=(1, 2), skip_driver=False):
    _build.build()
    cls = ics.cluster_batch(ncl, seed)
    pats = _patterns(cls, seed + 1, npat)
    variants = list(range(5)) if variants is None else variants
    sweep = []
    for v in variants:
        for gm in grid_muls:
            sec, inter, _ = force_calls(cls, v, gm, 0, pats, reps)
            sweep.append(dict(variant=v, grid_mul=gm, ms_per_call=1e3 * sec,
                              interactions_per_s=inter / sec))
    best = min(sweep, key=lambda r: r["ms_per_call"])
    v, gm = best["variant"], best["grid_mul"]
    modes = {}
    for mode, name in ((0, "graph"), (1, "plain"), (2, "per_cluster")):
        sec, inter, launches = force_calls(cls, v, gm, mode, pats, reps)
        modes[name] = dict(ms_per_call=1e3 * sec, interactions_per_s=inter / sec,
                           gflops_60=FLOPS * inter / sec / 1e9,
                           launches_per_call=launches / (1 + (reps + 1) * len(pats)))
    out = dict(workload="batch of %d Plummer clusters, N log-uniform [256, 16384], Salpeter, "
               "eps2=(4/N)^2, seed %d" % (ncl, seed),
               sum_n=int(sum(c["n"] for c in cls)), patterns=npat,
               tune_sweep=sweep, tuned=dict(variant=v, grid_mul=gm), force_calls=modes,
               speedup_graph_vs_per_cluster=modes["per_cluster"]["ms_per_call"]
               / modes["graph"]["ms_per_call"])
    if not skip_driver:
        out["driver"] = [driver(cls, v, gm, mode, t_end, eta) for mode in (0, 2)]
        out["driver_t_end"] = t_end
        out["driver_speedup_graph_vs_per_cluster"] = (out["driver"][1]["wall_s"]
                                                      / out["driver"][0]["wall_s"])
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--ncl", type=int, default=256)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--t-end", type=float, default=0.0625)
    ap.add_argument("--eta", type=float, default=0.01)
    ap.add_argument("--patterns", type=int, default=16)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--no-driver", action="store_true")
    a = ap.parse_args(argv)
    print(json.dumps(run(a.ncl, a.seed, a.t_end, a.eta, a.patterns, a.reps,
                         skip_driver=a.no_driver)))
    return 0


if __name__ == "__main__":
    sys.exit(main())
