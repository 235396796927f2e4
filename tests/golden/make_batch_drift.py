"""Write tests/golden/batch_drift.txt: for every cluster of the batch
workload (256 Plummer clusters, N log-uniform in [256, 16384], Salpeter
masses, eps2 = (4/N)^2, seed 1), the FP64 oracle's energy E0 and its relative
energy drift dE/E after its own 4th-order Hermite block-time-step
integration to t = 1/16 with eta = 0.01 (Sect. 2, Sect. 3.2).  Calls only
oracle/ and the shared input generators; run once, commit the output.

    python tests/golden/make_batch_drift.py
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_0902_4463_gb300 import ics  # noqa: E402

NCL, SEED, ETA, T_END = 256, 1, 0.01, 0.0625


def main():
    orc = oracle.default()
    cls = ics.cluster_batch(NCL, SEED)
    lines = ["# FP64 oracle, batch of %d clusters (seed %d), Hermite to t = %g, eta = %g"
             % (NCL, SEED, T_END, ETA),
             "# cluster n eps2 E0 dE_over_E nblocks nactive seconds"]
    t_all = time.time()
    for k, c in enumerate(cls):
        e0 = orc.energy(c["m"], c["x"], c["v"], c["eps2"])
        t0 = time.time()
        r = orc.hermite_run(c["m"], c["x"], c["v"], c["eps2"], ETA, T_END)
        assert r["err"] == 0 and r["t"] == T_END
        e1 = orc.energy(c["m"], r["x"], r["v"], c["eps2"])
        lines.append("%d %d %.17g %.17g %.6e %d %d %.1f" % (
            k, c["n"], c["eps2"], e0, (e1 - e0) / e0, r["nblocks"], r["nactive"],
            time.time() - t0))
    lines.append("# total seconds %.0f" % (time.time() - t_all))
    with open(os.path.join(HERE, "batch_drift.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
