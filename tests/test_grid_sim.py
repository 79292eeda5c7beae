"""The vectorised simulator used by the full-size GPU property checks agrees
with the node-by-node simulator written from eq. 2d_graph_dynamics."""
import numpy as np

from paper_2304_04980_gb300 import synth
from tests import grid_sim
from tests.test_oracle_pins import as_problem, simulate


def test_vectorised_simulator_matches_loop_simulator():
    for (K, N, T, n, m) in ((3, 5, 4, 2, 1), (4, 1, 3, 3, 2), (1, 4, 3, 2, 2)):
        g = synth.random_grid(K, N, T, n, m, seed=K * N)
        u = synth.random_vector((T, K * N, m), seed=1)
        w = synth.random_vector((T, K * N, n), seed=2)
        P = as_problem(g, w=w)
        ref = simulate(P, u, w)
        got = grid_sim.simulate(K, N, T, g.A_self, g.A_nbr, g.B, g.x0, u, w)
        assert np.allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
