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


# --------------------------------------------------------------------------
# the multi-right-hand-side solve (Algorithm 1 per right-hand side)
# --------------------------------------------------------------------------

SOLVE_SHAPES = [(5, 6, 9), (4, 5, 7), (9, 7, 33), (1, 1, 3), (8, 2, 12)]


def x0_block(g, nrhs, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((nrhs, g.nodes, g.n))


@pytest.mark.parametrize("shape", SOLVE_SHAPES, ids=["K%dN%dT%d" % s for s in SOLVE_SHAPES])
def test_multi_rhs_solve_matches_oracle(dev, shape):
    """Every right-hand side's costate, x and u against the oracle's dense
    solution for that initial state, its true residual within the
    tolerance, and a zero initial state solved in zero steps."""
    K, N, T = shape
    g = synth.random_grid(K, N, T, 4, 2, seed=700 + K * 7 + N * 3 + T)
    prob = lq().Problem.from_grid(g)
    nrhs = 32
    x0s = x0_block(g, nrhs, seed=K + N + T)
    x0s[5] = 0.0
    xt = torch.from_numpy(x0s).to(dev)
    x = torch.empty((nrhs, g.T + 1, g.nodes, g.n), dtype=torch.float64, device=dev)
    u = torch.empty((nrhs, g.T, g.nodes, g.m), dtype=torch.float64, device=dev)
    lam = torch.empty_like(x)
    out = prob.solve_multi_device(nrhs, xt, 1e-10, 2, 2, 5000, x=x, u=u, costate=lam)
    assert out["status"] == 0
    assert max(out["rel_residuals"]) <= 1e-10
    assert out["iterations"][5] == 0
    xh, uh, lh = x.cpu().numpy(), u.cpu().numpy(), lam.cpu().numpy()
    for r in (0, 5, 17, 31):
        ref = O.Oracle(O.Problem.from_arrays(g.K, g.N, g.T, g.n, g.m, *g.with_x0(x0s[r]).arrays())).solve(1e-12)
        scale = max(np.linalg.norm(ref.delta), 1e-300)
        assert np.linalg.norm(lh[r] - ref.delta) <= 1e-7 * scale + 1e-300
        assert np.linalg.norm(xh[r] - ref.x) <= 1e-7 * max(np.linalg.norm(ref.x), 1e-300) + 1e-300
        assert np.linalg.norm(uh[r] - ref.u) <= 1e-7 * max(np.linalg.norm(ref.u), 1e-300) + 1e-300
    prob.close()


def test_multi_rhs_solve_agrees_with_single_solves_and_affine(dev):
    """Fewer than 32 right-hand sides; the same solutions as single
    solves (FP64) within the tolerance's reach; boundary terms from
    lq2d_set_affine enter every right-hand side; iteration counts stay
    within a small factor of the single FP64 solves (TF32 preconditioner)."""
    lq2d = lq()
    g = synth.random_grid(7, 8, 25, 4, 2, seed=77)
    prob = lq2d.Problem.from_grid(g)
    w = synth.random_vector((g.T, g.nodes, g.n), seed=8) * 0.1
    prob.set_affine(w)
    nrhs = 7
    x0s = x0_block(g, nrhs, seed=3)
    out = prob.solve_multi_device(nrhs, torch.from_numpy(x0s).to(dev), 1e-10, 2, 2, 5000,
                                  costate=(lam := torch.empty((nrhs, g.T + 1, g.nodes, g.n), dtype=torch.float64,
                                                              device=dev)))
    assert out["status"] == 0 and len(out["iterations"]) == nrhs
    for r in range(nrhs):
        single = lq2d.Problem.from_grid(g.with_x0(x0s[r]))
        single.set_affine(w)
        s = single.solve(1e-12, 2, 2, 5000)
        ref = s["costate"]
        assert np.linalg.norm(lam[r].cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)
        assert out["iterations"][r] <= 2 * s["iterations"] + 10
        single.close()
    prob.close()


def test_multi_rhs_solve_limits_and_errors(dev):
    lq2d = lq()
    g = synth.random_grid(4, 4, 8, 4, 2, seed=9)
    prob = lq2d.Problem.from_grid(g)
    x0s = torch.from_numpy(x0_block(g, 4, seed=1)).to(dev)
    out = prob.solve_multi_device(4, x0s, 1e-12, 2, 2, 2)
    assert out["status"] == lq2d.ENOCONV
    for nrhs, tol, L in ((0, 1e-8, 2), (33, 1e-8, 2), (4, 0.0, 2), (4, 1e-8, 3)):
        with pytest.raises(lq2d.LQ2DError):
            prob.solve_multi_device(nrhs, x0s, tol, 2, L, 100)
    prob.close()


def test_multi_rhs_solve_full_size_bench_workload(dev):
    """K = N = 64, T = 100, 32 initial states (scaled Gaussian bumps at
    random centres): every right-hand side's true residual meets 1e-8 and
    four of them agree with single FP64 solves to 1e-6."""
    lq2d = lq()
    g = synth.workload("grid64_T100")
    rng = np.random.default_rng(5)
    ii, jj = np.meshgrid(np.arange(g.K), np.arange(g.N), indexing="ij")
    x0s = np.empty((32, g.nodes, g.n))
    for r in range(32):
        ci, cj = rng.uniform(0, g.K, 2)
        bump = np.exp(-((ii - ci) ** 2 + (jj - cj) ** 2) / (2 * (g.K / 8) ** 2)).ravel()
        x0s[r] = bump[:, None] * rng.uniform(0.5, 2.0, g.n)[None, :]
    prob = lq2d.Problem.from_grid(g)
    lam = torch.empty((32, g.T + 1, g.nodes, g.n), dtype=torch.float64, device=dev)
    out = prob.solve_multi_device(32, torch.from_numpy(x0s).to(dev), 1e-8, 2, 2, 5000, costate=lam)
    assert out["status"] == 0 and max(out["rel_residuals"]) <= 1e-8
    for r in (0, 9, 22, 31):
        single = lq2d.Problem.from_grid(g.with_x0(x0s[r]))
        ref = single.solve(1e-10, 2, 2, 5000)["costate"]
        assert np.linalg.norm(lam[r].cpu().numpy() - ref) <= 1e-6 * np.linalg.norm(ref)
        single.close()
    prob.close()
