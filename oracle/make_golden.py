"""Writes tests/golden/grid4_T20.json: the oracle's solution of the K=N=4,
n=2, m=1, T=20 workload (seed 0) at S = L = 2, tol 1e-10, with the
conditioning figures of Section V measured on it.

Run from the repository root:  python -m oracle.make_golden
The paper prints no worked example for this method, so every stored value
here comes from the oracle (test infrastructure), never from the CUDA path.
"""
import json
import os
import sys

import numpy as np
import scipy.linalg as sla

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import lq2d_oracle as O  # noqa: E402
from paper_2304_04980_gb300 import synth  # noqa: E402


def main():
    g = synth.workload("grid4_T20")
    P = O.Problem.from_arrays(g.K, g.N, g.T, g.n, g.m, *g.arrays())
    orc = O.Oracle(P)
    sol = orc.solve(1e-10, 2, 2)
    ref = orc.solve(1e-14, 2, 2)
    D = orc.Delta.toarray()
    ev = np.linalg.eigvalsh(D)
    DS = O.nbjm_closed_form(orc.splitting, 2, 2)
    evp = sla.eigh(D, np.linalg.inv(DS), eigvals_only=True)
    out = {
        "what": "oracle solution of the K=N=4, n=2, m=1, T=20 random-grid workload (seed 0)",
        "method": "Algorithm 1 (PCGM) with Algorithm 2 (NBJM) preconditioner, S=2, L=2",
        "written_by": "python -m oracle.make_golden",
        "K": g.K, "N": g.N, "T": g.T, "n": g.n, "m": g.m, "seed": 0,
        "tol": 1e-10, "S": 2, "L": 2,
        "iterations": sol.iterations,
        "rel_kkt": sol.rel_kkt,
        "cost": ref.cost,
        "kappa_delta": float(ev[-1] / ev[0]),
        "kappa_preconditioned": float(evp[-1] / evp[0]),
        "delta": ref.delta.ravel().tolist(),
        "x": ref.x.ravel().tolist(),
        "u": ref.u.ravel().tolist(),
    }
    path = os.path.join(ROOT, "tests", "golden", "grid4_T20.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=0)
    print("wrote", path, "iterations", sol.iterations, "cost", ref.cost)


if __name__ == "__main__":
    main()
