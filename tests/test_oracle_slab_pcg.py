"""Pins for the slab-by-slab oracle (oracle/slab_pcg.py), the form of the
oracle that reaches the K = N = 256, T = 200 grid: its splitting blocks,
Algorithm 2 and Algorithm 1 against the assembled oracle, whose masks of the
explicit Delta are pinned in test_oracle_pins.py (Riccati, dense KKT, the
Theorem's closed form).  The process-parallel evaluation must give the same
numbers as the serial one."""
import numpy as np
import pytest

from oracle import lq2d_oracle as O
from oracle import slab_pcg as SP
from paper_2304_04980_gb300 import synth

CASES = [(3, 4, 5, 2, 1), (4, 5, 6, 3, 2), (1, 3, 4, 2, 2), (2, 1, 3, 1, 1), (3, 5, 1, 2, 1), (4, 4, 2, 4, 2)]
IDS = ["K%dN%dT%dn%dm%d" % c for c in CASES]


def problem(shape, seed=0):
    K, N, T, n, m = shape
    g = synth.random_grid(K, N, T, n, m, seed=seed + sum(shape))
    return O.Problem.from_arrays(K, N, T, n, m, *g.arrays())


@pytest.mark.parametrize("shape", CASES, ids=IDS)
def test_slab_splitting_blocks_equal_the_masks_of_delta(shape):
    P = problem(shape)
    orc = O.Oracle(P)
    Sp = orc.splitting
    ss = SP.SlabSplitting(P)
    w = P.nodes * P.n
    for t in range(P.T + 1):
        sl = slice(t * w, (t + 1) * w)
        cb = ss.cls[SP.time_class(t, P.T)]
        for name, M in (("Psi", Sp.Psi), ("Phi", Sp.Phi), ("Omega", Sp.Omega)):
            got = getattr(cb, name).toarray()
            want = M[sl, sl].toarray()
            assert np.abs(got - want).max() <= 1e-13 * max(1.0, np.abs(want).max()), (name, t)
        if t >= 1:
            lo = slice((t - 1) * w, t * w)
            assert np.abs(ss.XiL.toarray() - Sp.Xi[sl, lo].toarray()).max() <= 1e-13
            assert np.abs(ss.XiU.toarray() - Sp.Xi[lo, sl].toarray()).max() <= 1e-13


@pytest.mark.parametrize("shape", CASES, ids=IDS)
@pytest.mark.parametrize("SL", [(1, 2), (2, 2), (3, 4)])
def test_slab_preconditioner_equals_algorithm2(shape, SL):
    P = problem(shape, seed=1)
    orc = O.Oracle(P)
    S, L = SL
    pre = orc.preconditioner(S, L)
    r = np.random.default_rng(3).standard_normal(P.dim_x)
    want = pre.apply(r)
    with SP.SlabOracle(P) as so:
        got = so.precondition(r, S, L)
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
        d = so.delta_apply(r)
        assert np.abs(d - orc.Delta @ r).max() <= 1e-13 * np.abs(d).max()


def test_slab_pcg_matches_the_assembled_oracle_and_the_parallel_form():
    P = problem((6, 5, 9, 4, 2), seed=2)
    ref = O.Oracle(P).solve(1e-11)
    with SP.SlabOracle(P) as so:
        res = so.solve(1e-11)
    assert res.converged and abs(res.iterations - ref.iterations) <= 1
    assert np.linalg.norm(res.delta - ref.delta.ravel()) <= 1e-9 * np.linalg.norm(ref.delta)
    with SP.SlabOracle(P, workers=3) as par:
        assert len(par.ranges) == 3
        r = np.random.default_rng(5).standard_normal(P.dim_x)
        with SP.SlabOracle(P) as ser:
            assert np.array_equal(par.precondition(r, 2, 2), ser.precondition(r, 2, 2))
            assert np.array_equal(par.delta_apply(r), ser.delta_apply(r))
        res2 = par.solve(1e-11)
    assert res2.iterations == res.iterations and np.array_equal(res2.delta, res.delta)
