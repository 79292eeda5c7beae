"""Multi-right-hand-side preconditioner on the tensor cores through the
C-ABI: q_r = D_S r_r for up to 32 right-hand sides at once (Algorithm 2,
Theorem posdef_preconditioner) against the oracle's D_S r for each of them.

The products use TF32 operands (an 11-bit significand, unit roundoff
2^-11 = 4.9e-4) with FP32 accumulation.  One sweep applies about 2K
products in sequence (forward and backward substitution over K pair-rows)
and S x L sweeps follow each other, so the bound below allows the rounding
of some tens of products: 2e-2 of the largest entry of D_S r."""
import numpy as np
import pytest

from oracle import lq2d_oracle as O
from paper_2304_04980_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TF32_BOUND = 2e-2


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


SHAPES = [(5, 6, 9), (4, 5, 7), (9, 7, 33), (3, 3, 4), (8, 2, 12), (1, 1, 3)]


def rhs_block(g, nrhs, seed):
    return np.stack([synth.random_vector((g.T + 1, g.nodes, g.n), seed=seed + r) for r in range(nrhs)])


@pytest.mark.parametrize("shape", SHAPES, ids=["K%dN%dT%d" % s for s in SHAPES])
@pytest.mark.parametrize("SL", [(2, 2), (1, 2), (3, 4)])
def test_multi_rhs_preconditioner_matches_oracle(dev, shape, SL):
    """Each right-hand side against the oracle's Algorithm 2, for ragged
    tiles of time steps, odd N (a one-column last pair), K = 1 and several
    (S, L)."""
    K, N, T = shape
    S, L = SL
    g = synth.random_grid(K, N, T, 4, 2, seed=600 + K * 7 + N * 3 + T)
    orc = O.Oracle(O.Problem.from_arrays(g.K, g.N, g.T, g.n, g.m, *g.arrays()))
    pre = orc.preconditioner(S, L)
    prob = lq().Problem.from_grid(g)
    nrhs = 32
    r = rhs_block(g, nrhs, seed=41)
    rt = torch.from_numpy(r).to(dev)
    q = torch.empty_like(rt)
    prob.apply_precond_multi_device(nrhs, S, L, rt, q)
    qh = q.cpu().numpy()
    worst = 0.0
    for k in range(nrhs):
        ref = pre.apply(r[k].ravel())
        err = np.abs(qh[k].ravel() - ref).max() / np.abs(ref).max()
        worst = max(worst, err)
    assert worst <= TF32_BOUND, worst
    prob.close()


def test_multi_rhs_counts_layout_and_rebuild(dev):
    """Fewer than 32 right-hand sides leave the rest of the output alone;
    a single right-hand side equals the first of a full panel; the operands
    are rebuilt after an update of the problem data."""
    lq2d = lq()
    g = synth.random_grid(6, 6, 11, 4, 2, seed=71)
    g2 = synth.random_grid(6, 6, 11, 4, 2, seed=72)
    prob = lq2d.Problem.from_grid(g)
    r = rhs_block(g, 32, seed=3)
    rt = torch.from_numpy(r).to(dev)
    q_all = torch.empty_like(rt)
    prob.apply_precond_multi_device(32, 2, 2, rt, q_all)
    q_one = torch.full_like(rt, 7.0)
    prob.apply_precond_multi_device(1, 2, 2, rt, q_one)
    assert torch.equal(q_one[0], q_all[0])
    assert bool((q_one[1:] == 7.0).all())
    q5 = torch.empty_like(rt[:5])
    prob.apply_precond_multi_device(5, 2, 2, rt[:5].contiguous(), q5)
    assert torch.equal(q5, q_all[:5])
    # new data: results follow the new problem
    prob.update_device(*[torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in g2.arrays()])
    q_new = torch.empty_like(rt)
    prob.apply_precond_multi_device(32, 2, 2, rt, q_new)
    ref = O.Oracle(O.Problem.from_arrays(g2.K, g2.N, g2.T, g2.n, g2.m, *g2.arrays())).preconditioner(2, 2)
    for k in (0, 31):
        want = ref.apply(r[k].ravel())
        assert np.abs(q_new[k].cpu().numpy().ravel() - want).max() <= TF32_BOUND * np.abs(want).max()
    prob.close()


def test_multi_rhs_rejects_bad_arguments(dev):
    lq2d = lq()
    g = synth.random_grid(4, 4, 5, 4, 2, seed=5)
    prob = lq2d.Problem.from_grid(g)
    r = torch.zeros((33, g.T + 1, g.nodes, 4), dtype=torch.float64, device=dev)
    q = torch.empty_like(r)
    for nrhs, S, L in ((0, 2, 2), (33, 2, 2), (2, 0, 2), (2, 2, 3)):
        with pytest.raises(lq2d.LQ2DError):
            prob.apply_precond_multi_device(nrhs, S, L, r, q)
    prob.close()
    g3 = synth.random_grid(4, 4, 5, 3, 2, seed=5)
    p3 = lq2d.Problem.from_grid(g3)
    r3 = torch.zeros((2, g3.T + 1, g3.nodes, 3), dtype=torch.float64, device=dev)
    with pytest.raises(lq2d.LQ2DError):
        p3.apply_precond_multi_device(2, 2, 2, r3, torch.empty_like(r3))
    p3.close()


def test_multi_rhs_full_size_bench_workload(dev):
    """K = N = 64, T = 100 with 32 right-hand sides: every one within the
    TF32 bound of the FP64 single-right-hand-side preconditioner (itself
    checked against the oracle), and D_S r_r . r_r > 0 (the Theorem)."""
    lq2d = lq()
    g = synth.workload("grid64_T100")
    prob = lq2d.Problem.from_grid(g)
    r = rhs_block(g, 32, seed=900)
    rt = torch.from_numpy(r).to(dev)
    q = torch.empty_like(rt)
    prob.apply_precond_multi_device(32, 2, 2, rt, q)
    for k in range(32):
        ref = torch.empty_like(rt[k])
        prob.apply_precond_device(2, 2, rt[k].contiguous(), ref)
        err = float((q[k] - ref).abs().max() / ref.abs().max())
        assert err <= TF32_BOUND, (k, err)
        assert float((q[k] * rt[k]).sum()) > 0.0
    prob.close()
