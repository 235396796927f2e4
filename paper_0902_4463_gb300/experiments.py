"""Paper-style experiments on one GPU (Sect. 3): equal-mass Plummer spheres
integrated with the library's Hermite block-time-step driver.

    python -m paper_0902_4463_gb300.experiments scaling --nmin 1024 --nmax 262144
    python -m paper_0902_4463_gb300.experiments eta --n 32768 131072 [--fp64]

* scaling (Sect. 3.1, wall-clock time, Gflop/s and mean block size against
  N): N = nmin .. nmax in powers of two, eta = 0.01, to t = 1/4.
* eta (Sect. 3.2, dE/E against the accuracy parameter): eta from 1e-4 to
  0.3 at the given N, to t = 1/4; with --fp64 also the all-FP64 GPU path,
  whose error floor is set by the integrator alone; with --noise R the DS
  runs choose their steps allowing for a relative force error R.

The paper does not state its softening; the runs here use eps = 4/N (the
close-encounter length of an N-body system in Henon units).  Energies are
evaluated with one all-FP64 force sweep.  Prints one JSON line per run and a
summary line.
"""
import argparse
import json
import sys

from . import hermite_run

ETAS = (1e-4, 3e-4, 1e-3, 3e-3, 1e-2, 3e-2, 0.1, 0.3)


def eps2_of(n):
    return (4.0 / n) ** 2


def one(n, eta, prec, seed=1, t_end=0.25, noise=0.0):
    r = hermite_run.run(n, seed, eps2_of(n), eta, t_end, prec, noise=noise)
    keep = ("n", "eta", "prec", "eps2", "t_end", "wall_s", "nblocks", "nactive", "mean_block",
            "interactions_per_s", "gflops_60", "dE_over_E", "synchronised", "force_noise")
    out = {k: r[k] for k in keep}
    out["force_s"] = r["profile"]["force_s"]
    out["host_s"] = r["profile"]["sched_s"] + r["profile"]["correct_s"]
    out["wall_per_time_unit_s"] = r["wall_s"] / t_end
    return out


def scaling(nmin, nmax, fp64_max=0, seed=1):
    rows = []
    n = nmin
    while n <= nmax:
        rows.append(one(n, 0.01, "ds", seed))
        print(json.dumps(rows[-1]), flush=True)
        if n <= fp64_max:
            rows.append(one(n, 0.01, "fp64", seed))
            print(json.dumps(rows[-1]), flush=True)
        n *= 2
    return rows


def eta_sweep(ns, fp64=False, seed=1, etas=ETAS, noise=0.0):
    rows = []
    for n in ns:
        for eta in etas:
            for prec in (("ds", "fp64") if fp64 else ("ds",)):
                rows.append(one(n, eta, prec, seed, noise=noise if prec == "ds" else 0.0))
                print(json.dumps(rows[-1]), flush=True)
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="what", required=True)
    s = sub.add_parser("scaling")
    s.add_argument("--nmin", type=int, default=1024)
    s.add_argument("--nmax", type=int, default=262144)
    s.add_argument("--fp64-max", type=int, default=0,
                   help="also run the all-FP64 path up to this N")
    e = sub.add_parser("eta")
    e.add_argument("--n", type=int, nargs="+", default=[32768, 131072])
    e.add_argument("--fp64", action="store_true")
    e.add_argument("--etas", type=float, nargs="+", default=list(ETAS))
    e.add_argument("--noise", type=float, default=0.0,
                   help="DS runs: relative force error the time-step choice allows for")
    a = ap.parse_args(argv)
    if a.what == "scaling":
        rows = scaling(a.nmin, a.nmax, a.fp64_max)
    else:
        rows = eta_sweep(a.n, a.fp64, etas=a.etas, noise=a.noise)
    print(json.dumps({"summary": a.what, "runs": len(rows)}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
