"""Write the oracle regression fixture l4_beta2_first_sweeps.json.

The plain-method case: L=4 (N=16), t=1, U=4, beta=2, dtau=0.1 (M=20), half
filling (8 up + 8 down worldlines), Philox seed 0.  The values are the oracle's own
(FP64) after 3 sweeps: the anchor slices, the filter log-weights of each sweep and the
final worldlines and field.  This script calls only oracle/; the fixture locks the
oracle's arithmetic against accidental change.  It is not a paper value: the paper
prints no worked example.
Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

PARAMS = dict(L=4, t=1.0, U=4.0, beta=2.0, dtau=0.1, filling=1.0, seed=0)
SWEEPS = 3


def compute():
    p = PARAMS
    ch = oracle.Chain(p["L"], p["t"], p["U"], p["beta"], p["dtau"], p["filling"], p["seed"])
    out = {"params": p, "sweeps": SWEEPS, "anchors": [], "logw": []}
    for _ in range(SWEEPS):
        r = ch.sweep()
        out["anchors"].append(int(r["anchor"]))
        out["logw"].append([[float(v) for v in row] for row in r["logw"]])
    out["x"] = ch.x.tolist()
    out["s"] = ch.s.tolist()
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "l4_beta2_first_sweeps.json"), "w") as f:
        json.dump(compute(), f, indent=1)
        f.write("\n")
