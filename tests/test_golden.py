"""The stored oracle fixture for the K=N=4, T=20 workload still matches the
oracle, and the fixture itself satisfies the KKT conditions."""
import json
import os

import numpy as np

from oracle import lq2d_oracle as O
from paper_2304_04980_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "grid4_T20.json")


def test_golden_fixture_matches_oracle():
    ref = json.load(open(GOLDEN))
    g = synth.workload("grid4_T20")
    P = O.Problem.from_arrays(g.K, g.N, g.T, g.n, g.m, *g.arrays())
    orc = O.Oracle(P)
    sol = orc.solve(ref["tol"], ref["S"], ref["L"])
    assert sol.iterations == ref["iterations"]
    delta = np.array(ref["delta"])
    assert np.linalg.norm(sol.delta.ravel() - delta) <= 1e-8 * np.linalg.norm(delta)
    x, u = O.recover(orc.S, delta)
    assert O.kkt_residual(orc.S, x, u, delta) < 1e-12
    assert np.allclose(x, ref["x"], atol=1e-12) and np.allclose(u, ref["u"], atol=1e-12)
    assert abs(O.cost(orc.S, x, u) - ref["cost"]) < 1e-10 * ref["cost"]
