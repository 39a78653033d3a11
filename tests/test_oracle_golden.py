"""The oracle reproduces its stored small-case output (written by
tests/golden/make_golden.py from the oracle alone) on this platform."""
import json
import os

import numpy as np

import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_small.json")


def test_oracle_matches_stored_output(oracle_lib):
    data = json.load(open(GOLDEN))
    for case in data["cases"]:
        c = W.Contract(**case["contract"])
        mean, se, per = oracle_lib.greeks(data["seed"], c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma,
                                          c.construction, c.N, c.R)
        assert np.allclose(per, case["per_replicate"], rtol=1e-13, atol=1e-15)
        assert np.allclose(mean, case["mean"], rtol=1e-13, atol=1e-15)
        pts = oracle_lib.point_values(data["seed"], c.type, c.d, c.K, c.T, c.S0, c.r, c.sigma,
                                      c.construction, 1, 5, 3)
        assert np.allclose(pts, case["points_rep1_k5_8"], rtol=1e-13, atol=1e-15)
