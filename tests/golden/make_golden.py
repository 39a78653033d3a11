"""Write tests/golden/oracle_small.json from the CPU oracle only.

The stored values are the oracle's own output for a few small seeded cases;
they guard the oracle against unnoticed changes and against platform drift
(the GPU machine is Arm, the development box x86).  Run from the repository root:
    python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as W  # noqa: E402

CASES = [
    W.small_arith(),
    W.Contract(W.BINARY, 9, 105.0, 0.5, 100.0, 0.03, 0.3, 2 ** 10, 4, W.BB),
    W.Contract(W.LOOKBACK, 33, 95.0, 2.0, 100.0, 0.07, 0.25, 2 ** 10, 4, W.PCA),
    W.Contract(W.GEOMETRIC, 64, 100.0, 1.0, 100.0, 0.05, 0.2, 2 ** 9, 4, W.BB),
]


def main():
    out = []
    for c in CASES:
        mean, se, per = oracle.greeks(W.SCRAMBLE_SEED, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma,
                                      c.construction, c.N, c.R)
        pts = oracle.point_values(W.SCRAMBLE_SEED, c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma,
                                  c.construction, 1, 5, 3)
        out.append({"contract": c.__dict__, "mean": mean.tolist(), "se": se.tolist(),
                    "per_replicate": per.tolist(), "points_rep1_k5_8": pts.tolist()})
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_small.json")
    with open(path, "w") as f:
        json.dump({"source": "oracle/qmccpw_oracle.c via tests/golden/make_golden.py",
                   "seed": W.SCRAMBLE_SEED, "cases": out}, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
