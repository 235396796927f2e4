"""Batch workload: 256 independent Plummer clusters, N log-uniform in
[256, 16384], Salpeter masses, eps2 = (4/N)^2 (ics.cluster_batch).

    python -m paper_0902_4463_gb300.batch_run --ncl 256 --seed 1 --t-end 0.0625

Two measurements, both printed as one JSON line:

* force-only batch calls (Sect. 2: one force call per block step, here for
  every cluster at once) on seeded uneven active sets: per cluster
  ni = max(1, N >> u), u uniform in 0 .. floor(log2 N), a fifth of the
  clusters idle per call.  The native schedule autotuner picks the
  schedule on these patterns; then each call is timed end to end (host
  staging, launch, wait, results in mapped memory) as one CUDA-graph
  replay, as plain launches and as one launch sequence per cluster, and
  every one-class schedule is timed for comparison;
* the Hermite batch driver (every cluster its own block scheduler, one batch
  force call per batch step) to t_end: the default schedule, then the
  schedule its autotuner picks from the active sets of its first 64 batch
  steps, in graph mode and with per-cluster launches.

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


def _make_batch(cls, sched=None):
    b = g6.G6Batch([c["n"] for c in cls])
    if sched is not None:
        b.set_schedule(*sched)
    for k, c in enumerate(cls):
        b.set_j(k, c["m"], c["x"], c["v"])
        b.set_i(k, c["x"], c["v"])
    return b


def _eps2_t(cls):
    return np.array([c["eps2"] for c in cls]), np.zeros(len(cls))


def force_calls(cls, sched, mode, patterns, reps):
    """Mean seconds per batch call and interactions per call."""
    b = _make_batch(cls, sched)
    try:
        eps2, t = _eps2_t(cls)
        n = np.array([c["n"] for c in cls])
        b.calc(t, eps2, n, mode)                 # staging, graph capture, warm-up
        for p in patterns:
            b.calc(t, eps2, p, mode)
        l0 = b.launch_count()
        t0 = time.perf_counter()
        for _ in range(reps):
            for p in patterns:
                b.calc(t, eps2, p, mode)
        sec = (time.perf_counter() - t0) / (reps * len(patterns))
        launches = (b.launch_count() - l0) / (reps * len(patterns))
        inter = float(np.mean([np.dot(p.astype(np.float64), n) for p in patterns]))
        return sec, inter, launches
    finally:
        b.close()


def tune_on(cls, patterns, reps):
    """Native schedule autotuner on the given active-set patterns."""
    b = _make_batch(cls)
    try:
        eps2, t = _eps2_t(cls)
        return b.autotune(np.stack(patterns), eps2, t, reps)
    finally:
        b.close()


def driver_patterns(cls, eta, steps):
    """Active-set patterns of the driver's first batch steps, and the
    schedule its own autotuner picks from them."""
    sim = g6.G6HBatchSim([(c["m"], c["x"], c["v"]) for c in cls],
                         [c["eps2"] for c in cls], eta)
    try:
        for _ in range(steps):
            if sim.step(1.0) == 0:
                break
        return sim.autotune(2)
    finally:
        sim.close()


def driver(cls, sched, mode, t_end, eta):
    sim = g6.G6HBatchSim([(c["m"], c["x"], c["v"]) for c in cls],
                         [c["eps2"] for c in cls], eta, mode=mode)
    try:
        if sched is not None:
            sim.set_schedule(sched)
        sim.set_timing(True)
        t0 = time.perf_counter()
        sim.run(t_end)
        wall = time.perf_counter() - t0
        st = sim.stats()
        gpu_ms, ncalls = sim.timing()
        ok = bool(np.all(sim.state()["t"] == t_end))
    finally:
        sim.close()
    return dict(mode=mode, schedule=sched, wall_s=wall, batch_steps=st["nsteps"],
                nactive=st["nactive"], interactions=st["interactions"],
                sec_gpu=st["sec_gpu"], sec_host=st["sec_host"],
                gpu_event_s=gpu_ms / 1e3, gpu_event_us_per_call=1e3 * gpu_ms / max(1, ncalls),
                interactions_per_s=st["interactions"] / wall,
                gflops_60=FLOPS * st["interactions"] / wall / 1e9,
                us_per_batch_step=1e6 * wall / max(1, st["nsteps"]),
                mean_active_per_cluster_step=st["nactive"] / max(1, st["nsteps"]) / len(cls),
                synchronised=ok)


def run(ncl=256, seed=1, t_end=0.0625, eta=0.01, npat=16, reps=3, skip_driver=False):
    _build.build()
    cls = ics.cluster_batch(ncl, seed)
    pats = _patterns(cls, seed + 1, npat)
    sched, ms = tune_on(cls, pats, reps)
    modes = {}
    for mode, name in ((0, "graph"), (1, "plain"), (2, "per_cluster")):
        sec, inter, launches = force_calls(cls, sched, mode, pats, reps)
        modes[name] = dict(ms_per_call=1e3 * sec, interactions_per_s=inter / sec,
                           gflops_60=FLOPS * inter / sec / 1e9, launches_per_call=launches)
    one = {}
    for v in range(8):
        sec, inter, _ = force_calls(cls, (v, 2, 0, -1, 1), 0, pats, reps)
        one[v] = 1e3 * sec
    out = dict(workload="batch of %d Plummer clusters, N log-uniform [256, 16384], Salpeter, "
               "eps2=(4/N)^2, seed %d" % (ncl, seed),
               sum_n=int(sum(c["n"] for c in cls)), patterns=npat,
               tuned_schedule=sched, tuned_ms=ms, one_class_ms_gm2=one, force_calls=modes,
               speedup_graph_vs_per_cluster=modes["per_cluster"]["ms_per_call"]
               / modes["graph"]["ms_per_call"])
    if not skip_driver:
        dsched, dms = driver_patterns(cls, eta, 64)
        out["driver_tuned_schedule"] = dsched
        out["driver_tuned_ms"] = dms
        out["driver"] = [driver(cls, None, 0, t_end, eta), driver(cls, dsched, 0, t_end, eta),
                         driver(cls, dsched, 2, t_end, eta)]
        out["driver_t_end"] = t_end
        out["driver_speedup_graph_vs_per_cluster"] = (out["driver"][2]["wall_s"]
                                                      / out["driver"][1]["wall_s"])
    return out


def driver_steps(ncl, seed, eta, steps, mode=0):
    """A few batch steps of the driver with the default schedule (the
    command that kernel profiles of the batch path run)."""
    _build.build()
    cls = ics.cluster_batch(ncl, seed)
    sim = g6.G6HBatchSim([(c["m"], c["x"], c["v"]) for c in cls],
                         [c["eps2"] for c in cls], eta, mode=mode)
    try:
        sim.set_timing(True)
        for _ in range(steps):
            if sim.step(1.0) == 0:
                break
        st = sim.stats()
        gpu_ms, calls = sim.timing()
    finally:
        sim.close()
    return dict(steps=st["nsteps"], nactive=st["nactive"], interactions=st["interactions"],
                gpu_event_us_per_call=1e3 * gpu_ms / max(1, calls))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--ncl", type=int, default=256)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--t-end", type=float, default=0.0625)
    ap.add_argument("--eta", type=float, default=0.01)
    ap.add_argument("--patterns", type=int, default=16)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--no-driver", action="store_true")
    ap.add_argument("--driver-steps", type=int, default=0,
                    help="only run this many driver batch steps (profiling command)")
    a = ap.parse_args(argv)
    if a.driver_steps:
        print(json.dumps(driver_steps(a.ncl, a.seed, a.eta, a.driver_steps)))
        return 0
    print(json.dumps(run(a.ncl, a.seed, a.t_end, a.eta, a.patterns, a.reps,
                         skip_driver=a.no_driver)))
    return 0


if __name__ == "__main__":
    sys.exit(main())
