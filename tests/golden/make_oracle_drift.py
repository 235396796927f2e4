"""Write tests/golden/oracle_drift.txt: the FP64 oracle's relative energy drift
dE/E = (E1 - E0)/E0 (Sect. 3.2) for the Plummer workloads of the parity tests,
integrated with the oracle's own 4th-order Hermite block-time-step scheme.
Calls only oracle/ and the shared input generators; run once, commit output.

    python tests/golden/make_oracle_drift.py [--quick]
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_0902_4463_gb300 import ics  # noqa: E402

CASES = [
    # name, n, seed, eps2, eta, t_end
    ("plummer_n1024", 1024, 1, 1e-4, 0.01, 0.25),
    ("plummer_n32768_t0.25", 32768, 2, 1e-5, 0.01, 0.25),
    ("plummer_n32768_t1", 32768, 2, 1e-5, 0.01, 1.0),
]


def main():
    quick = "--quick" in sys.argv
    orc = oracle.default()
    out = os.path.join(HERE, "oracle_drift.txt")
    lines = ["# FP64 oracle energy drift, Hermite block steps (Sect. 2, Sect. 3.2)",
             "# name n seed eps2 eta t_end dE_over_E nblocks nactive seconds"]
    for name, n, seed, eps2, eta, t_end in CASES:
        if quick and n > 1024:
            continue
        m, x, v = ics.plummer(n, seed)
        e0 = orc.energy(m, x, v, eps2)
        t0 = time.time()
        r = orc.hermite_run(m, x, v, eps2, eta, t_end)
        dt = time.time() - t0
        assert r["err"] == 0 and r["t"] == t_end
        e1 = orc.energy(m, r["x"], r["v"], eps2)
        lines.append("%s %d %d %g %g %g %.6e %d %d %.1f" % (
            name, n, seed, eps2, eta, t_end, (e1 - e0) / e0, r["nblocks"], r["nactive"], dt))
        print(lines[-1], flush=True)
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
