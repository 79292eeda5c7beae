"""Two-ended solve of Phi_bar in the NBJM sweeps (n = 4, K >= 4).

The per-(column pair, time step) SPD solve with Phi_bar (Algorithm 2; the
block-tridiagonal matrix along the pair-rows of Section III) can be done
from both ends at once: a forward block-Cholesky pass over the top half of
the pair-rows, one over the bottom half in reversed order, and a 2x2 block
interface system between them.  The result is the same linear map as the
one-ended solve up to rounding, so both are compared with the oracle's
preconditioner (FP64: 1e-11 relative; FP32 operands: 1e-4, the mixed
precision bound of the other FP32 tests) and with each other.  Shapes cover
the smallest K that splits (4), odd K (unequal halves), odd N (one-column
last pair), T = 1 and grids of several ragged tiles.
"""
import numpy as np
import pytest

from oracle import lq2d_oracle as O
from paper_2304_04980_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHAPES = [  # K, N, T, n, m
    (4, 4, 20, 4, 2),
    (5, 3, 9, 4, 2),
    (6, 7, 12, 4, 1),
    (7, 5, 6, 4, 2),
    (9, 7, 33, 4, 2),
    (16, 3, 5, 4, 2),
    (4, 1, 3, 4, 2),
    (12, 9, 1, 4, 2),
]
IDS = ["K%dN%dT%dn%dm%d" % s for s in SHAPES]
SL = [(1, 2), (2, 2), (3, 4)]


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_04980_gb300 import build
    build.build()
    return torch.device("cuda:0")


def lq():
    from paper_2304_04980_gb300 import lq2d
    return lq2d


def grid_for(shape, seed=0):
    K, N, T, n, m = shape
    return synth.random_grid(K, N, T, n, m, seed=400 + seed + 7 * K + 3 * N + T + n)


def oracle_for(g):
    return O.Oracle(O.Problem.from_arrays(g.K, g.N, g.T, g.n, g.m, *g.arrays()))


def tdev(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)


def rel_err(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def apply(prob, S, L, r, dev):
    q = torch.empty_like(tdev(r, dev))
    prob.apply_precond_device(S, L, tdev(r, dev), q)
    return q.cpu().numpy().ravel()


@pytest.mark.parametrize("shape", SHAPES, ids=IDS)
def test_fp64_two_ended_matches_oracle(dev, shape):
    lq2d = lq()
    g = grid_for(shape)
    orc = oracle_for(g)
    prob = lq2d.Problem.from_grid(g)
    assert prob.get_option(lq2d.OPT_TWISTED) == 1  # the default for n = 4, K >= 4
    r = synth.random_vector((g.T + 1, g.nodes, g.n), seed=5)
    for S, L in SL:
        ref = orc.preconditioner(S, L).apply(r.ravel())
        prob.set_option(lq2d.OPT_TWISTED, 0)
        one = apply(prob, S, L, r, dev)
        for thr in (32, 64):
            prob.set_option(lq2d.OPT_SWEEP_THREADS, thr)
            prob.set_option(lq2d.OPT_TWISTED, 1)
            assert prob.get_option(lq2d.OPT_TWISTED) == 1
            got = apply(prob, S, L, r, dev)
            assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max(), (thr, S, L)
            assert np.abs(got - one).max() <= 1e-11 * np.abs(one).max(), (thr, S, L)
            prob.set_option(lq2d.OPT_TWISTED, 0)
    prob.close()


@pytest.mark.parametrize("shape", SHAPES, ids=IDS)
def test_fp32_two_ended_matches_oracle(dev, shape):
    lq2d = lq()
    g = grid_for(shape, seed=1)
    orc = oracle_for(g)
    prob = lq2d.Problem.from_grid(g)
    prob.set_precision(1)
    prob.set_option(lq2d.OPT_SWEEP_STEPS, 0)
    r = synth.random_vector((g.T + 1, g.nodes, g.n), seed=6)
    for S, L in SL:
        ref = orc.preconditioner(S, L).apply(r.ravel())
        for thr in (32, 64):
            prob.set_option(lq2d.OPT_SWEEP_THREADS, thr)
            prob.set_option(lq2d.OPT_TWISTED, 1)
            assert prob.get_option(lq2d.OPT_TWISTED) == 1
            got = apply(prob, S, L, r, dev)
            assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max(), (thr, S, L)
            prob.set_option(lq2d.OPT_TWISTED, 0)
            one = apply(prob, S, L, r, dev)
            assert np.abs(got - one).max() <= 1e-4 * np.abs(one).max(), (thr, S, L)
    prob.close()


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("shape", [SHAPES[1], SHAPES[4]], ids=[IDS[1], IDS[4]])
def test_two_ended_solve_matches_oracle(dev, shape, mode):
    lq2d = lq()
    g = grid_for(shape, seed=2)
    ref = oracle_for(g).solve(1e-12, 2, 2, max_iter=5000)
    prob = lq2d.Problem.from_grid(g)
    prob.set_precision(mode)
    if mode:
        prob.set_option(lq2d.OPT_SWEEP_STEPS, 0)
    prob.set_option(lq2d.OPT_SWEEP_THREADS, 64)
    prob.set_option(lq2d.OPT_TWISTED, 1)
    tol = 1e-12 if mode == 0 else 1e-10
    out = prob.solve(tol, 2, 2, 20000)
    assert out["status"] == 0
    bound = 1e-8 if mode == 0 else 1e-6
    assert rel_err(out["costate"], ref.delta) <= bound
    assert rel_err(out["x"], ref.x) <= bound
    assert rel_err(out["u"], ref.u) <= bound
    prob.close()


def test_two_ended_follows_updates_and_small_grids(dev):
    """A data update refreshes the two-ended arrays; below K = 4 the option is
    accepted and the sweep stays one-ended; the bulk-copy FP32 schedules and
    widths above 64 report one-ended."""
    lq2d = lq()
    g = grid_for(SHAPES[2], seed=3)
    g2 = grid_for(SHAPES[2], seed=4)
    prob = lq2d.Problem.from_grid(g)
    prob.set_option(lq2d.OPT_TWISTED, 1)
    r = synth.random_vector((g.T + 1, g.nodes, g.n), seed=7)
    prob.update(*g2.arrays())
    ref = oracle_for(g2).preconditioner(2, 2).apply(r.ravel())
    got = apply(prob, 2, 2, r, dev)
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()
    prob.set_precision(1)
    prob.set_option(lq2d.OPT_SWEEP_STEPS, 4)
    assert prob.get_option(lq2d.OPT_TWISTED) == 0
    prob.set_option(lq2d.OPT_SWEEP_STEPS, 0)
    assert prob.get_option(lq2d.OPT_TWISTED) == 1
    prob.set_option(lq2d.OPT_SWEEP_THREADS, 128)
    assert prob.get_option(lq2d.OPT_TWISTED) == 0
    prob.set_option(lq2d.OPT_SWEEP_THREADS, 64)
    got = apply(prob, 2, 2, r, dev)
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()
    prob.close()

    small = grid_for((3, 4, 6, 4, 2))
    p3 = lq2d.Problem.from_grid(small)
    p3.set_option(lq2d.OPT_TWISTED, 1)
    assert p3.get_option(lq2d.OPT_TWISTED) == 0
    r3 = synth.random_vector((small.T + 1, small.nodes, small.n), seed=8)
    ref3 = oracle_for(small).preconditioner(2, 2).apply(r3.ravel())
    got3 = apply(p3, 2, 2, r3, dev)
    assert np.abs(got3 - ref3).max() <= 1e-11 * np.abs(ref3).max()
    p3.close()


def test_autotune_includes_two_ended(dev):
    lq2d = lq()
    g = grid_for((12, 8, 16, 4, 2), seed=5)
    orc = oracle_for(g)
    r = synth.random_vector((g.T + 1, g.nodes, g.n), seed=9)
    ref = orc.preconditioner(2, 2).apply(r.ravel())
    for mode, tol in ((0, 1e-11), (1, 1e-4)):
        prob = lq2d.Problem.from_grid(g)
        prob.set_precision(mode)
        thr, ms = prob.autotune(2, 2, reps=2)
        assert ms > 0 and thr in (32, 64, 128, 256)
        assert prob.get_option(lq2d.OPT_SWEEP_THREADS) == thr
        assert prob.get_option(lq2d.OPT_TWISTED) in (0, 1)
        got = apply(prob, 2, 2, r, dev)
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
        prob.close()
