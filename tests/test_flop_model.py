"""The algorithmic flop model behind bench.py's roofline, against the
structure of the oracle's explicit matrices.

Per sweep (Algorithm 2), the model counts: the band solves of every
Phi_bar_{v,t} block for t >= 1 (Section IV-B), theta_0 = Q tau at t = 0,
and the products with Omega~ and Xi~.  Here each term is counted a second
way, from the matrices the oracle assembles:
  * a banded solve with a Cholesky factor touches the factor's envelope,
    and the factor fills in exactly inside the matrix's profile, so row r
    of a block costs e_r = r - (first nonzero column of row r) multiply-adds
    plus one pivot scaling, forward and backward, with the unknowns in the
    kernels' order (pair-row, column, component), which is the oracle's
    natural order inside a (v, t) block;
  * a product with Omega~ or Xi~ costs one multiply-add per nonzero;
  * at t = 0, Phi_bar is Q^-1 node by node and theta_0 = Q tau costs one
    multiply-add per entry of that block diagonal.
Each multiply-add is 2 flops, each scaling 1."""
import dataclasses

import numpy as np
import pytest

import bench
from oracle import lq2d_oracle as O
from paper_2304_04980_gb300 import synth


def nonzeros(M):
    return int(np.count_nonzero(M.toarray()))


def dense_weights(g, seed):
    """The grid with random SPD Q and Q_T blocks, so that no block of the
    model is structurally sparser than the kernels treat it (with Q = I,
    Phi_bar at t = 0 would be diagonal)."""
    rng = np.random.default_rng(seed)

    def spd(scale):
        a = rng.standard_normal((g.nodes, g.n, g.n))
        return np.einsum("pij,pkj->pik", a, a) + scale * np.eye(g.n)

    return dataclasses.replace(g, Q=spd(g.n), Q_T=spd(2 * g.n))


# odd and even N (a one-column last pair), K = 1 and 2 (no second band),
# n = 1..4
SHAPES = [(5, 6, 3, 2), (6, 5, 4, 3), (4, 7, 2, 4), (1, 4, 3, 2), (2, 3, 2, 1), (3, 1, 2, 2)]


@pytest.mark.parametrize("K,N,T,n", SHAPES, ids=["K%dN%dT%dn%d" % s for s in SHAPES])
def test_sweep_flop_model_matches_the_oracle_matrices(K, N, T, n):
    g = dense_weights(synth.random_grid(K, N, T, n, 2, seed=40 + K + N + n), seed=K * N)
    orc = O.Oracle(O.Problem.from_arrays(g.K, g.N, g.T, g.n, g.m, *g.arrays()))
    Sp = orc.splitting
    t, _, _, _ = O.labels(orc.P)
    band = 0
    t0 = 0
    for grp in Sp.groups:
        blk = Sp.Phi[grp][:, grp].toarray()
        if t[grp[0]] == 0:
            t0 += 2 * int(np.count_nonzero(blk))
            continue
        for r in range(len(grp)):
            e = r - int(np.flatnonzero(blk[r, : r + 1])[0])
            band += 2 * (2 * e + 1)
    fl = bench.sweep_flops(g)
    assert fl["plain"] == band + t0
    assert fl["omega"] - fl["plain"] == 2 * nonzeros(Sp.Omega)
    assert fl["xi"] - fl["plain"] == 2 * nonzeros(Sp.Xi)
    # the block solves dominate every sweep but the tiny ones
    if K >= 4:
        assert band > 2 * nonzeros(Sp.Omega)


def test_t0_block_is_node_diagonal_and_omega_vanishes_there():
    """The two facts the model's t = 0 term rests on (reading A17)."""
    g = dense_weights(synth.random_grid(4, 5, 3, 2, 1, seed=7), seed=8)
    orc = O.Oracle(O.Problem.from_arrays(g.K, g.N, g.T, g.n, g.m, *g.arrays()))
    Sp = orc.splitting
    t, i, j, _ = O.labels(orc.P)
    Phi = Sp.Phi.tocoo()
    at0 = (t[Phi.row] == 0) & (Phi.data != 0)
    assert np.all(i[Phi.row[at0]] == i[Phi.col[at0]]) and np.all(j[Phi.row[at0]] == j[Phi.col[at0]])
    Om = Sp.Omega.tocoo()
    assert not np.any((t[Om.row] == 0) & (Om.data != 0))
