"""Benchmark of the direct-summation Hermite force path (arXiv:0902.4463).

Workload: Plummer sphere, N = 2^20 equal masses, eps2 = 1e-6, every j-particle
last updated at t_j = 0 and predicted to t_blk = 2^-10, every particle active
(m = N).  One step is one pass of the whole hot path on that block:
j-memory update of the m corrected particles, prediction of all N
j-particles (Eq. 1, Eq. 2), force with DS separations (Eq. 3) plus nearest
neighbour, and the FP64 reduction of the partial forces (Sect. 2.1-2.3).

Metric: interactions/s = m * N / step time, and Gflop/s at 60 flop per pair
(Sect. 2.3 / Sect. 3.1 convention).  The all-FP64 kernel is timed on a subset
of the active block (its rate is flat in m) for the DS-over-FP64 speed-up.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--n N] [--m M] [--sweep] [--fp64-m M] [--no-cpu-baseline]
  python bench.py --latency --n N [--reps R]        per-call cost of small block steps
  python bench.py --experiment scaling|eta [...]     paper-style Hermite runs (Sect. 3)
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FLOPS_PER_PAIR = 60          # Sect. 2.3 and Sect. 3.1 footnote
FLOPS_PER_PAIR_DS = 66       # Sect. 2.3: with the DS separations of Eq. 3
FP32_LANES_PER_SM = 128      # FP32 FMA lanes per Blackwell SM
METRIC = "interactions/s & Gflop/s (60 flop/pair) N=2^20: FP32+DS vs FP64 on 1 GB300"
EPS2 = 1e-6
T_BLK = 2.0 ** -10
SEED = 3
CID = 0
KERNEL_SRC = os.path.join(ROOT, "paper_0902_4463_gb300", "csrc", "g6gb_kernels.cu")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_force_ds_plummer_n262144_and_n1048576.md")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1 << 20)
    ap.add_argument("--m", type=int, default=0, help="active block size (0: N)")
    ap.add_argument("--fp64-m", type=int, default=4096)
    ap.add_argument("--sweep", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--tune", default="", help="run the autotuner first and write its table here")
    ap.add_argument("--tune-file", default="", help="load an autotuner table before timing")
    ap.add_argument("--prec", default="ds", choices=["ds", "ds_x64"],
                    help="DS predictor: the paper's DS + SP add (ds) or an FP64 add (ds_x64)")
    ap.add_argument("--variant", type=int, default=-1)
    ap.add_argument("--grid", type=int, default=0)
    ap.add_argument("--latency", action="store_true",
                    help="per-call cost of small block steps through the GRAPE calls at --n")
    ap.add_argument("--reps", type=int, default=200, help="--latency: repetitions per size")
    ap.add_argument("--experiment", choices=["scaling", "eta"], default=None,
                    help="paper-style Hermite runs (Sect. 3): wall clock, Gflop/s and mean "
                         "block size against N, or dE/E against eta")
    ap.add_argument("--nmin", type=int, default=1024)
    ap.add_argument("--nmax", type=int, default=262144)
    ap.add_argument("--fp64-max", type=int, default=0)
    ap.add_argument("--ns", type=int, nargs="+", default=[32768, 131072])
    ap.add_argument("--etas", type=float, nargs="+",
                    default=[1e-4, 3e-4, 1e-3, 3e-3, 1e-2, 3e-2, 0.1, 0.3])
    ap.add_argument("--fp64", action="store_true", help="--experiment eta: also all-FP64 runs")
    ap.add_argument("--noise", type=float, default=0.0,
                    help="--experiment eta: relative force error the DS step choice allows for")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, ws, device):
    """The largest x over all ranks (x itself when ws == 1)."""
    if ws <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_rate(units_per_rank, seconds_max, ws):
    """Whole-job throughput of ws replicas that each processed units_per_rank
    units, timed by the slowest rank."""
    return ws * float(units_per_rank) / seconds_max


def workload(n, m):
    from paper_0902_4463_gb300 import ics
    st = ics.taylor_state(n, SEED, T_BLK, dt_levels=None)
    act = np.arange(n) if m == n else np.sort(ics.permutation(n, SEED)[:m])
    return st, act


def jrecords(st, sel):
    from paper_0902_4463_gb300 import g6gb as g6
    rec = np.zeros(sel.size, dtype=g6.JREC)
    rec["x"] = st["x0"][sel]
    rec["v"] = st["v0"][sel]
    rec["a2"] = st["a0"][sel] / 2.0
    rec["j6"] = st["j0"][sel] / 6.0
    rec["mass"] = st["m"][sel]
    rec["tj"] = st["tj"][sel]
    rec["address"] = sel
    rec["index"] = sel
    return rec


def irecords(st, act):
    from paper_0902_4463_gb300 import g6gb as g6
    rec = np.zeros(act.size, dtype=g6.IREC)
    rec["x"] = st["x0"][act]
    rec["v"] = st["v0"][act]
    rec["index"] = act
    return rec


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.lines = []

    def __enter__(self):
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[4 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_traffic():
    """DRAM bytes per force launch from the committed ncu capture, if it was
    taken on the current kernel source (else None)."""
    try:
        rec = {}
        for line in open(TRAFFIC_FILE):
            if ":" in line and not line.startswith(("|", "#", " ")):
                k, v = line.split(":", 1)
                rec[k.strip()] = v.strip()
        sha = hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()
        if rec.get("kernel_source_sha256") == sha:
            return int(rec["traffic_bytes_per_launch_full"])
    except (OSError, ValueError, KeyError):
        pass
    return None


def cpu_oracle_rate(st, act, target_s=12.0, max_i=None):
    """Oracle (FP64, OpenMP over i) on a bounded sample of the active block
    against all N j-particles predicted by the oracle.  Returns a dict."""
    import oracle
    orc = oracle.default()
    n = st["m"].shape[0]
    t0 = time.perf_counter()
    xp, vp = orc.predict(st["x0"], st["v0"], st["a0"], st["j0"], st["tj"], T_BLK)
    t_pred = time.perf_counter() - t0
    idx = np.arange(n)
    ms = 8
    t = 0.0
    while True:
        sel = act[:ms]
        t0 = time.perf_counter()
        res = orc.force(st["x0"][sel], st["v0"][sel], sel, xp, vp, st["m"], idx, EPS2)
        t = time.perf_counter() - t0
        if t >= target_s / 4 or ms >= act.size or (max_i and ms >= max_i):
            break
        ms = min(act.size, ms * max(2, int(target_s / 4 / max(t, 1e-3))))
        if max_i:
            ms = min(ms, max_i)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return dict(rate=ms * n / t, seconds=t, m_sample=int(ms), cores=int(cores),
                t_predict=t_pred, result=res, sel=act[:ms])


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    n = args.n
    m = args.m or n
    st, act = workload(n, m)
    # size one step to about 60 s / (steps + warmup) of CPU work
    per_step = max(2.0, min(30.0, 90.0 / max(1, args.steps + args.warmup)))
    probe = cpu_oracle_rate(st, act, target_s=per_step)
    ms_i = probe["m_sample"]
    import oracle
    orc = oracle.default()
    xp, vp = orc.predict(st["x0"], st["v0"], st["a0"], st["j0"], st["tj"], T_BLK)
    idx = np.arange(n)
    sel = act[:ms_i]
    for _ in range(args.warmup):
        orc.force(st["x0"][sel], st["v0"][sel], sel, xp, vp, st["m"], idx, EPS2)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        orc.predict(st["x0"], st["v0"], st["a0"], st["j0"], st["tj"], T_BLK)
        orc.force(st["x0"][sel], st["v0"][sel], sel, xp, vp, st["m"], idx, EPS2)
    dt = (time.perf_counter() - t0) / args.steps
    rate = ms_i * n / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "interactions/s",
        "n_gpus": 0, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "gflops_60": rate * FLOPS_PER_PAIR / 1e9,
        "config": {"workload": "plummer_N%d_full_block_sweep" % n, "n": n, "m": m,
                   "eps2": EPS2, "t_blk": T_BLK, "seed": SEED},
        "cpu_baseline": {"value": rate, "unit": "interactions/s", "cores": probe["cores"],
                         "kind": "oracle",
                         "sample": "%d of the %d active i-particles against all %d j "
                                   "(FP64 oracle, OpenMP over i) per step" % (ms_i, m, n)},
        "e2e": {"value": rate, "unit": "interactions/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_latency(args):
    """Per-call cost of one block step through the GRAPE calling sequence
    (Sect. 2.1, 2.5): for block sizes m = 1 .. 4096 against n j-particles
    (uniform in a unit cube, eps2 = 1e-4), each repetition updates the m
    j-records (g6x_set_j_particles), sets a new block time (g6_set_ti, so the
    j-particles are predicted again), starts the force (g6calc_firsthalf) and
    waits for it (g6calc_lasthalf2).  One JSON line per m: the host wall time
    of each call (microseconds, mean over the repetitions after 20 warm-up
    ones; the calls go through ctypes, which adds about a microsecond each),
    then, from a second pass with the library's CUDA-event timing on (every
    kernel then launched on its own), the device time of each phase, and the
    launch configuration."""
    from paper_0902_4463_gb300 import build as gbuild
    gbuild.build()
    from paper_0902_4463_gb300 import g6gb as g6
    n, reps = args.n, args.reps
    rng = np.random.default_rng(12345)
    x = rng.uniform(size=(n, 3))
    v = rng.uniform(-0.5, 0.5, size=(n, 3))
    m = np.full(n, 1.0 / n)
    z = np.zeros((n, 3))
    idx = np.arange(n, dtype=np.int32)
    lib = g6.lib()
    P = g6._p
    g6.g6x_open_ex(CID, n, 4096)
    try:
        g6.g6x_set_j_particles(CID, idx, idx, 0.0, m, z, z, v, x)
        acc, jerk, pot = np.empty((4096, 3)), np.empty((4096, 3)), np.empty(4096)
        nnb = np.empty(4096, dtype=np.int32)
        t = 0.0
        for mm in (1, 16, 64, 256, 1024, 4096):
            sel = np.ascontiguousarray(idx[:mm])
            tj = np.zeros(mm)
            mj = np.ascontiguousarray(m[:mm])
            xs, vs = np.ascontiguousarray(x[:mm]), np.ascontiguousarray(v[:mm])
            zs = np.ascontiguousarray(z[:mm])

            # the argument pointers are made once, so that each timed call
            # pays only the ctypes call itself
            p_sel, p_tj, p_mj, p_zs, p_vs, p_xs = (P(a) for a in (sel, tj, mj, zs, vs, xs))
            p_acc, p_jerk, p_pot, p_nnb = (P(a) for a in (acc, jerk, pot, nnb))

            def one():
                nonlocal t
                t += 2.0 ** -20
                tj[:] = t - 2.0 ** -20
                t0 = time.perf_counter()
                lib.g6x_set_j_particles(CID, mm, p_sel, p_sel, p_tj, p_mj, p_zs, p_zs, p_vs,
                                        p_xs)
                t1 = time.perf_counter()
                lib.g6_set_ti(CID, t)
                lib.g6calc_firsthalf(CID, n, mm, p_sel, p_xs, p_vs, None, None, None, 1e-4,
                                     None)
                t2 = time.perf_counter()
                rc = lib.g6calc_lasthalf2(CID, n, mm, None, None, None, 1e-4, None, p_acc,
                                          p_jerk, p_pot, p_nnb)
                t3 = time.perf_counter()
                if rc < 0:
                    raise g6.G6Error(rc, "g6calc_lasthalf2")
                return t1 - t0, t2 - t1, t3 - t2

            for _ in range(20):
                one()
            tot = np.zeros(3)
            for _ in range(reps):
                tot += one()
            host = tot / reps * 1e6
            g6.g6x_set_timing(CID, True)
            for _ in range(reps):
                one()
            ms, cnt = g6.g6x_get_timing(CID)
            g6.g6x_set_timing(CID, False)
            cfg = g6.g6x_last_config(CID)
            dev = [ms[k] / max(1, cnt[k]) * 1e3 for k in range(4)]
            print(json.dumps({"n": n, "m": mm, "set_j_us": host[0], "firsthalf_us": host[1],
                              "lasthalf_us": host[2], "total_us": float(host.sum()),
                              "device_us": {"store_predict": dev[0] + dev[1], "force": dev[2],
                                            "reduce": dev[3]},
                              "launches_per_step": sum(int(c) for c in cnt) / reps,
                              "config": cfg}), flush=True)
    finally:
        g6.g6_close(CID)
    return 0


def run_experiment(args):
    """Paper-style experiments on one GPU (Sect. 3) with the library's Hermite
    block-time-step driver on equal-mass Plummer spheres, to t = 1/4:
    `scaling` -- wall clock, Gflop/s and mean block size against N (powers of
    two from --nmin to --nmax, eta = 0.01; all-FP64 runs up to --fp64-max);
    `eta` -- dE/E against the accuracy parameter at each N of --ns (with
    --fp64 also the all-FP64 path; --noise R lets the DS step choice allow for
    a relative force error R).  The paper does not state its softening; these
    runs use eps = 4/N.  Energies come from one all-FP64 force sweep.  One JSON
    line per run."""
    from paper_0902_4463_gb300 import hermite_run

    def one(n, eta, prec, noise=0.0):
        r = hermite_run.run(n, 1, (4.0 / n) ** 2, eta, 0.25, prec, noise=noise)
        keep = ("n", "eta", "prec", "eps2", "t_end", "wall_s", "nblocks", "nactive",
                "mean_block", "interactions_per_s", "gflops_60", "dE_over_E", "synchronised",
                "force_noise")
        out = {k: r[k] for k in keep}
        out["force_s"] = r["profile"]["force_s"]
        out["host_s"] = r["profile"]["sched_s"] + r["profile"]["correct_s"]
        print(json.dumps(out), flush=True)

    if args.experiment == "scaling":
        n = args.nmin
        while n <= args.nmax:
            one(n, 0.01, "ds")
            if n <= args.fp64_max:
                one(n, 0.01, "fp64")
            n *= 2
    else:
        for n in args.ns:
            for eta in args.etas:
                one(n, eta, "ds", args.noise)
                if args.fp64:
                    one(n, eta, "fp64")
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.latency:
        return run_latency(args)
    if args.experiment:
        return run_experiment(args)
    ws, rank, local = dist_env()
    import torch
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_0902_4463_gb300 import build as gbuild
    gbuild.build()
    from paper_0902_4463_gb300 import g6gb as g6

    n = args.n
    m = args.m or n
    st, act = workload(n, m)
    jrec_all = jrecords(st, np.arange(n))
    jrec_act = jrecords(st, act)
    irec = irecords(st, act)

    g6.g6x_use_torch_allocator()
    g6.g6x_open_ex(CID, n, max(m, 1))
    # a dedicated (non-legacy) stream: the library and the timing events
    # below both run on it
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    g6.g6x_set_stream(CID, stream.cuda_stream)
    if args.variant >= 0 or args.grid > 0:
        g6.g6x_set_variant(CID, args.variant, args.grid)
    if args.tune_file:
        g6.g6x_load_tuning(args.tune_file)
    DS_MODE = g6.G6X_PREC_DS_X64 if args.prec == "ds_x64" else g6.G6X_PREC_DS
    g6.g6x_set_precision(CID, DS_MODE)

    def to_dev(a):
        return torch.from_numpy(a.view(np.uint8).copy()).to(dev)

    d_jall = to_dev(jrec_all)
    d_jact = to_dev(jrec_act)
    d_irec = to_dev(irec)
    d_out = torch.empty(m * g6.OUT.itemsize, dtype=torch.uint8, device=dev)
    g6.g6x_set_j_dev(CID, n, d_jall.data_ptr())
    tuned = None
    if args.tune:
        t0 = time.perf_counter()
        tuned = {"sizes": g6.g6x_autotune(CID, n, m, args.tune), "file": args.tune,
                 "seconds": round(time.perf_counter() - t0, 1)}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count

    def step(mm, d_j, d_i, d_o):
        g6.g6x_set_j_dev(CID, mm, d_j.data_ptr())
        g6.g6x_calc_dev(CID, T_BLK, n, mm, d_i.data_ptr(), EPS2, 0, d_o.data_ptr())

    def timed(mm, d_j, d_i, d_o, steps, warmup, sampler=None, median=False):
        for _ in range(warmup):
            step(mm, d_j, d_i, d_o)
        g6.g6x_sync(CID)
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        g6.g6x_set_timing(CID, True)
        l0 = g6.g6x_launch_count(CID)
        times = []
        ctx = sampler if sampler is not None else _Null()
        with ctx:
            for _ in range(steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                step(mm, d_j, d_i, d_o)
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        launches = g6.g6x_launch_count(CID) - l0
        ms_ph, cnt = g6.g6x_get_timing(CID)
        g6.g6x_set_timing(CID, False)
        g6.g6x_sync(CID)
        step_ms = float(np.median(times)) if median else sum(times) / steps
        return step_ms, ms_ph, cnt, launches

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid)
    ms_step, ms_ph, cnt, launches = timed(m, d_jact, d_irec, d_out, args.steps, args.warmup,
                                          sampler)
    cfg = g6.g6x_last_config(CID)
    ms_step = max_over_ranks(ms_step, ws, dev)
    pairs = float(m) * n
    value = replica_rate(pairs, ms_step * 1e-3, ws)
    force_ms = ms_ph[2] / max(1, cnt[2])
    achieved = FLOPS_PER_PAIR * pairs / (force_ms * 1e-3) / 1e12
    clocks = sampler.summary()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    fmax = float(peaks.get("sm_max_mhz") or 2070.0)
    peak = sms * FP32_LANES_PER_SM * 2 * fmax * 1e6 / 1e12
    out_main = d_out.cpu().numpy().view(g6.OUT)
    # measured packed-FP32 and FP64 FMA rates (outside the timed region),
    # beside the derived peak the fraction is taken against and as the
    # denominator of the all-FP64 kernel's fraction
    probe_tf, probe_ms = g6.g6x_fp32_probe(10000)
    probe64_tf, probe64_ms = g6.g6x_fp64_probe(400)

    # the legs below take the built-in launch choice for their own precision
    if args.variant >= 0 or args.grid > 0:
        g6.g6x_set_variant(CID, -1, 0)
    # all-FP64 kernel on a subset of the block (its rate is flat in m)
    m64 = min(args.fp64_m, m)
    d_i64 = to_dev(irec[:m64])
    d_j64 = to_dev(jrec_act[:m64])
    d_o64 = torch.empty(m64 * g6.OUT.itemsize, dtype=torch.uint8, device=dev)
    g6.g6x_set_precision(CID, g6.G6X_PREC_FP64)
    ms64, ph64, c64, _ = timed(m64, d_j64, d_i64, d_o64, 2, 1)
    out64 = d_o64.cpu().numpy().view(g6.OUT)
    g6.g6x_set_precision(CID, DS_MODE)
    msds, phds, cds, _ = timed(m64, d_j64, d_i64, d_o64, 3, 2)
    rate64 = m64 * n / (ph64[2] / max(1, c64[2]) * 1e-3)
    rateds = m64 * n / (phds[2] / max(1, cds[2]) * 1e-3)
    # accuracy ablation: separations by the full DS subtraction
    g6.g6x_set_precision(CID, g6.G6X_PREC_DS_DSSUB)
    _, phss, css, _ = timed(m64, d_j64, d_i64, d_o64, 3, 2)
    g6.g6x_set_precision(CID, DS_MODE)
    ratess = m64 * n / (phss[2] / max(1, css[2]) * 1e-3)

    sweep = None
    if args.sweep:
        sweep = []
        mm = 16
        while mm <= m:
            d_is = to_dev(irec[:mm])
            d_js = to_dev(jrec_act[:mm])
            d_os = torch.empty(mm * g6.OUT.itemsize, dtype=torch.uint8, device=dev)
            # the median of 10 CUDA-event timed steps after 3 warm-up steps;
            # the phase times are means over the same 10 steps
            mss, phs, cs, _ = timed(mm, d_js, d_is, d_os, 10, 3, median=True)
            c = g6.g6x_last_config(CID)
            fms = phs[2] / max(1, cs[2])
            sweep.append({"m": mm, "ms_step": round(mss, 5),
                          "interactions_per_s": mm * n / (mss * 1e-3),
                          "force_interactions_per_s": mm * n / (fms * 1e-3),
                          "force_frac_fp32_peak": FLOPS_PER_PAIR * mm * n / (fms * 1e-3) / 1e12 / peak,
                          "predict_ms": phs[1] / max(1, cs[1]),
                          "scatter_ms": phs[0] / max(1, cs[0]),
                          "force_ms": fms, "reduce_ms": phs[3] / max(1, cs[3]),
                          "variant": c["variant"],
                          "grid": c["grid"]})
            mm *= 2

    # end to end through the public GRAPE-6 calls with host buffers
    e2e = None
    if not args.no_e2e:
        xi, vi = np.ascontiguousarray(irec["x"]), np.ascontiguousarray(irec["v"])
        idx_i = np.ascontiguousarray(irec["index"])
        addr = np.ascontiguousarray(jrec_act["address"])
        tj = np.ascontiguousarray(jrec_act["tj"])
        mass = np.ascontiguousarray(jrec_act["mass"])
        j6 = np.ascontiguousarray(jrec_act["j6"])
        a2 = np.ascontiguousarray(jrec_act["a2"])
        vj = np.ascontiguousarray(jrec_act["v"])
        xj = np.ascontiguousarray(jrec_act["x"])
        lib = g6.lib()
        P = g6.C.c_void_p

        def api_step():
            lib.g6x_set_j_particles(CID, m, g6._p(addr), g6._p(addr), g6._p(tj), g6._p(mass),
                                    g6._p(j6), g6._p(a2), g6._p(vj), g6._p(xj))
            lib.g6_set_ti(CID, T_BLK)
            lib.g6calc_firsthalf(CID, n, m, g6._p(idx_i), g6._p(xi), g6._p(vi), None, None,
                                 None, EPS2, None)
            rc = lib.g6calc_lasthalf2(CID, n, m, None, None, None, EPS2, None, g6._p(acc),
                                      g6._p(jerk), g6._p(pot), g6._p(nnb))
            if rc < 0:
                raise g6.G6Error(rc, "g6calc_lasthalf2")
            # host corrector and next time steps of the block (row a6)
            rc = lib.g6h_correct_block(m, T_BLK, g6._p(tj), g6._p(dt_cur), 0.01, 2.0 ** -4,
                                       2.0 ** -40, g6._p(xc), g6._p(vc), g6._p(a0), g6._p(j0),
                                       g6._p(acc), g6._p(jerk), g6._p(dt_new))
            if rc < 0:
                raise g6.G6Error(rc, "g6h_correct_block")

        acc = np.empty((m, 3))
        jerk = np.empty((m, 3))
        pot = np.empty(m)
        nnb = np.empty(m, dtype=np.int32)
        a0 = np.ascontiguousarray(st["a0"][act])
        j0 = np.ascontiguousarray(st["j0"][act])
        dt_cur = np.full(m, T_BLK)
        dt_new = np.empty(m)
        xc, vc = xi.copy(), vi.copy()
        k2 = max(1, min(args.steps, 3))
        api_step()
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for _ in range(k2):
            api_step()
        torch.cuda.synchronize()
        t_e2e = (time.perf_counter() - t0) / k2
        t_e2e = max_over_ranks(t_e2e, ws, dev)
        e2e = {"value": replica_rate(pairs, t_e2e, ws), "unit": "interactions/s",
               "h2d_bytes_per_step": int(m * (g6.JREC.itemsize + g6.IREC.itemsize)),
               "d2h_bytes_per_step": int(m * g6.OUT.itemsize + 4),
               "ms_per_step": t_e2e * 1e3,
               "api": "g6x_set_j_particles + g6_set_ti + g6calc_firsthalf + g6calc_lasthalf2"
                      " + g6h_correct_block (host corrector and time steps)"}

    cpu = None
    accuracy = None
    if rank == 0 and not args.no_cpu_baseline:
        r = cpu_oracle_rate(st, act[:m64], target_s=12.0, max_i=m64)
        oa, oj, op, onn, onr = r["result"]
        k = r["m_sample"]

        def errs(o):
            ea = np.linalg.norm(o["acc"][:k] - oa, axis=1) / np.linalg.norm(oa, axis=1)
            ej = np.linalg.norm(o["jerk"][:k] - oj, axis=1) / np.linalg.norm(oj, axis=1)
            ep = np.abs(o["pot"][:k] - op) / np.abs(op)
            return {"acc_rel_median": float(np.median(ea)), "acc_rel_max": float(ea.max()),
                    "jerk_rel_median": float(np.median(ej)), "jerk_rel_max": float(ej.max()),
                    "pot_rel_median": float(np.median(ep)), "pot_rel_max": float(ep.max()),
                    "nn_index_match": float(np.mean(o["nnb"][:k] == onn))}

        # the DS results of the main block are indexed by act; the sample is act[:k]
        accuracy = {"sample_i": int(k), "ds": errs(out_main[:k]), "fp64": errs(out64[:k])}
        cpu = {"value": r["rate"], "unit": "interactions/s", "cores": r["cores"],
               "kind": "oracle",
               "sample": "%d of the %d active i-particles against all %d j-particles "
                         "(FP64 oracle, OpenMP over i), %.1f s" % (k, m, n, r["seconds"])}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "interactions/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+ds", "data": "synthetic",
            "gflops_60": value * FLOPS_PER_PAIR / 1e9,
            "gflops_66": value * FLOPS_PER_PAIR_DS / 1e9,
            "config": {"workload": "plummer_N%d_full_block_sweep" % n, "n": n, "m": m,
                       "eps2": EPS2, "t_blk": T_BLK, "seed": SEED, "predictor": args.prec,
                       "l2": "256 MiB buffer written between timed steps",
                       "parallelism": "replicas" if ws > 1 else "single_gpu",
                       "kernel": cfg},
            "phases_ms_per_step": {"scatter": ms_ph[0] / max(1, cnt[0]),
                                   "predict": ms_ph[1] / max(1, cnt[1]),
                                   "force": force_ms, "reduce": ms_ph[3] / max(1, cnt[3])},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": kernel_traffic(),
                         "kernel": "k_force_ds (K2)",
                         "peak_basis": "%d SMs x %d FP32 lanes x 2 flop x %.0f MHz (max SM clock)"
                                       % (sms, FP32_LANES_PER_SM, fmax),
                         "frac_at_sampled_clock": (achieved / (sms * FP32_LANES_PER_SM * 2 *
                                                   clocks["sm_mhz"] * 1e6 / 1e12)
                                                   if clocks.get("sm_mhz") else None),
                         "fp32_probe": {"tflops": probe_tf, "ms": probe_ms,
                                        "of_derived_peak": probe_tf / peak,
                                        "force_frac_of_probe": achieved / probe_tf,
                                        "how": "g6x_fp32_probe: packed FP32x2 FMA chains, "
                                               "8 CTAs x 256 threads per SM"}},
            "fp64": {"m": m64, "force_interactions_per_s": rate64,
                     "gflops_60": rate64 * FLOPS_PER_PAIR / 1e9,
                     "peak_tflops": probe64_tf,
                     "peak_basis": "g6x_fp64_probe: FP64 FMA chains, 8 CTAs x 256 threads per SM "
                                   "(measured)",
                     "frac": rate64 * FLOPS_PER_PAIR / 1e12 / probe64_tf,
                     "ds_force_interactions_per_s_same_m": rateds,
                     "speedup_ds_over_fp64": rateds / rate64,
                     "speedup_ds_over_fp64_at_m_n": (pairs / (force_ms * 1e-3)) / rate64,
                     "speedup_basis_at_m_n": "DS force rate of the timed m = N step over the "
                                             "FP64 rate at m = %d (the FP64 kernel is bound by "
                                             "its pipe, its rate flat in m)" % m64},
            "ablation_full_ds_subtraction": {"m": m64, "force_interactions_per_s": ratess,
                                             "eq3_force_interactions_per_s": rateds,
                                             "eq3_speedup": rateds / ratess},
            "accuracy": accuracy,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks,
            "gpu_launches": int(launches),
        }
        if sweep is not None:
            line["sweep"] = sweep
        if tuned is not None:
            line["autotune"] = tuned
        print(json.dumps(line))
    g6.g6_close(CID)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


if __name__ == "__main__":
    sys.exit(main())
