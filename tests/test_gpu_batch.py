"""Batched solve (many uneven problems, one graph launch) through the C-ABI:
each problem's result equals its own single solve bit for bit (same
kernels, same order, deterministic reductions) and matches the oracle."""
import numpy as np
import pytest

from oracle import lq2d_oracle as O
from paper_2304_04980_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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


def small_batch(count=10):
    return synth.batch_grids(count, seed=17, K_range=(2, 9), N_range=(1, 9), T_range=(2, 14))


def costate_of(prob, g, dev):
    lam = torch.empty((g.T + 1, g.nodes, g.n), dtype=torch.float64, device=dev)
    prob.get_solution_device(costate=lam)
    return lam.cpu().numpy()


def test_batch_equals_single_solves_and_oracle(dev):
    lq2d = lq()
    grids = small_batch()
    probs = [lq2d.Problem.from_grid(g) for g in grids]
    for p in probs:  # the persistent loop's sweeps are one-sided
        p.set_option(lq2d.OPT_TWISTED, 0)
    batch = lq2d.Batch(probs)
    out = batch.solve(1e-11, 2, 2, 5000)
    assert out["status"] == 0 and all(s == 0 for s in out["statuses"])
    batched = [costate_of(p, g, dev) for p, g in zip(probs, grids)]
    for idx, (p, g) in enumerate(zip(probs, grids)):
        single = p.solve(1e-11, 2, 2, 5000)
        assert single["iterations"] == out["iterations"][idx]
        assert np.array_equal(single["costate"], batched[idx])
    for idx in (0, len(grids) - 1):
        g = grids[idx]
        ref = O.Oracle(O.Problem.from_arrays(g.K, g.N, g.T, g.n, g.m, *g.arrays())).solve(1e-12)
        rel = np.linalg.norm(batched[idx] - ref.delta) / np.linalg.norm(ref.delta)
        assert rel <= 1e-8
    batch.close()


def test_batch_rebuilds_and_sees_updated_data(dev):
    lq2d = lq()
    grids = small_batch(6)
    probs = [lq2d.Problem.from_grid(g) for g in grids]
    batch = lq2d.Batch(probs)
    a = batch.solve(1e-10, 2, 2, 5000)
    b = batch.solve(1e-6, 2, 2, 5000)          # new tolerance: graph rebuilt
    assert all(x <= y for x, y in zip(b["iterations"], a["iterations"]))
    probs[2].set_precision(1)                  # new mode for one problem: rebuilt
    c = batch.solve(1e-10, 2, 2, 5000)
    assert c["status"] == 0
    # new initial state for one problem, same graph
    g = grids[3]
    x0 = synth.random_vector(g.x0.shape, seed=99)
    g2 = g.with_x0(x0)
    probs[3].update_device(*[torch.from_numpy(np.ascontiguousarray(v)).to(dev) for v in g2.arrays()])
    d = batch.solve(1e-10, 2, 2, 5000)
    assert d["status"] == 0
    ref = O.Oracle(O.Problem.from_arrays(g2.K, g2.N, g2.T, g2.n, g2.m, *g2.arrays())).solve(1e-12)
    lam = costate_of(probs[3], g2, dev)
    assert np.linalg.norm(lam - ref.delta) <= 1e-7 * np.linalg.norm(ref.delta)
    batch.close()


def test_batch_reports_non_convergence_per_problem(dev):
    lq2d = lq()
    grids = small_batch(4)
    probs = [lq2d.Problem.from_grid(g) for g in grids]
    batch = lq2d.Batch(probs)
    out = batch.solve(1e-12, 2, 2, 2)
    assert out["status"] == lq2d.ENOCONV
    assert all(s == lq2d.ENOCONV for s in out["statuses"])
    assert all(it == 2 for it in out["iterations"])
    batch.close()


WIDTH_SHAPES = [(3, 5, 9, 1, 1), (4, 4, 20, 2, 1), (5, 6, 10, 3, 2), (9, 7, 33, 4, 2), (4, 5, 7, 5, 2),
                (3, 4, 37, 6, 3), (4, 3, 6, 7, 2), (6, 3, 7, 8, 3)]


@pytest.mark.parametrize("shape", WIDTH_SHAPES, ids=["K%dN%dT%dn%dm%d" % s for s in WIDTH_SHAPES])
@pytest.mark.parametrize("mode", [0, 1])
def test_sweep_widths_match_oracle(dev, shape, mode):
    """Every sweep tile width (32, 64, 128 and 256 threads: tiles of 2 to 128
    time steps per CTA depending on n, with ragged last tiles at these sizes)
    gives the same preconditioner up to rounding, and the default width the
    same solution."""
    lq2d = lq()
    K, N, T, n, m = shape
    g = synth.random_grid(K, N, T, n, m, seed=400 + 7 * K + 3 * N + T + n)
    orc = O.Oracle(O.Problem.from_arrays(g.K, g.N, g.T, g.n, g.m, *g.arrays()))
    prob = lq2d.Problem.from_grid(g)
    prob.set_precision(mode)
    r = synth.random_vector((g.T + 1, g.nodes, g.n), seed=5)
    rt = torch.from_numpy(r).to(dev)
    ref = orc.preconditioner(2, 2).apply(r.ravel())
    bound = (1e-11 if mode == 0 else 1e-4) * np.abs(ref).max()
    out = prob.solve(1e-10, 2, 2, 5000)
    assert out["status"] == 0
    lam = orc.solve(1e-12).delta
    assert np.linalg.norm(out["costate"] - lam) <= 1e-7 * np.linalg.norm(lam)
    for thr in (32, 64, 128, 256):
        prob.set_option(lq2d.OPT_SWEEP_THREADS, thr)
        q = torch.empty_like(rt)
        prob.apply_precond_device(2, 2, rt, q)
        assert np.abs(q.cpu().numpy().ravel() - ref).max() <= bound, thr
        assert prob.stats()["sweep_threads"] == thr


def test_autotune_picks_a_width_and_keeps_results(dev):
    lq2d = lq()
    g = synth.random_grid(16, 12, 40, 4, 2, seed=21)
    prob = lq2d.Problem.from_grid(g)
    base = prob.solve(1e-10, 2, 2, 5000)
    thr, ms = prob.autotune(2, 2, 3)
    assert thr in (32, 64, 128, 256) and ms > 0
    assert prob.stats()["sweep_threads"] == thr
    out = prob.solve(1e-10, 2, 2, 5000)
    assert out["status"] == 0
    assert np.linalg.norm(out["costate"] - base["costate"]) <= 1e-8 * np.linalg.norm(base["costate"])
    prob.set_precision(1)
    thr32, _ = prob.autotune(2, 2, 3)
    assert thr32 in (32, 64, 128, 256)
    assert prob.solve(1e-10, 2, 2, 5000)["status"] == 0
    with pytest.raises(lq2d.LQ2DError):
        prob.set_option(lq2d.OPT_SWEEP_THREADS, 100)
    with pytest.raises(lq2d.LQ2DError):
        prob.autotune(2, 3, 1)


def test_persistent_loop_equals_chains_single_solves_and_oracle(dev):
    """The persistent batched loop (one launch per kernel of a PCG step for
    every problem, work pulled from a device queue) gives each problem the
    result of its own single solve with the same sweep width and one-sided
    sweeps, bit for bit, and the one-chain-per-problem graph gives the same;
    uneven K, N, T (odd N, K = 1, N = 1 included).  With the two-ended solve
    (the single solves' default) the chains match the oracle."""
    lq2d = lq()
    grids = synth.batch_grids(12, seed=23, K_range=(1, 11), N_range=(1, 12), T_range=(1, 30))
    probs = [lq2d.Problem.from_grid(g) for g in grids]
    for p in probs:
        p.set_option(lq2d.OPT_TWISTED, 0)
    batch = lq2d.Batch(probs)
    for width in (32, 128, 64):
        batch.set_option(lq2d.BATCH_THREADS, width)
        out = batch.solve(1e-11, 2, 2, 5000)
        assert batch.get_option(lq2d.BATCH_USES_PERSISTENT) == 1
        assert out["status"] == 0
        persistent = [costate_of(p, g, dev) for p, g in zip(probs, grids)]
        for idx, (p, g) in enumerate(zip(probs, grids)):
            p.set_option(lq2d.OPT_SWEEP_THREADS, width)
            single = p.solve(1e-11, 2, 2, 5000)
            assert single["iterations"] == out["iterations"][idx]
            assert np.array_equal(single["costate"], persistent[idx])
    batch.set_option(lq2d.BATCH_PERSISTENT, 0)
    chains = batch.solve(1e-11, 2, 2, 5000)
    assert batch.get_option(lq2d.BATCH_USES_PERSISTENT) == 0
    assert chains["iterations"] == out["iterations"]
    for p, g, lam in zip(probs, grids, persistent):
        assert np.array_equal(costate_of(p, g, dev), lam)
    for p in probs:
        p.set_option(lq2d.OPT_TWISTED, 1)
    chains2 = batch.solve(1e-11, 2, 2, 5000)
    assert chains2["status"] == 0
    for idx in (0, 5, len(grids) - 1):
        g = grids[idx]
        ref = O.Oracle(O.Problem.from_arrays(g.K, g.N, g.T, g.n, g.m, *g.arrays())).solve(1e-12)
        assert np.linalg.norm(persistent[idx] - ref.delta) <= 1e-8 * np.linalg.norm(ref.delta)
        assert np.linalg.norm(costate_of(probs[idx], g, dev) - ref.delta) <= 1e-8 * np.linalg.norm(ref.delta)
    batch.close()


def test_batch_autotune_picks_a_width_and_the_batch_still_solves(dev):
    lq2d = lq()
    grids = synth.batch_grids(8, seed=29, K_range=(4, 16), N_range=(4, 16), T_range=(8, 40))
    probs = [lq2d.Problem.from_grid(g) for g in grids]
    batch = lq2d.Batch(probs)
    threads, ms = batch.autotune(2, 2, 2)
    assert threads in (32, 64, 128) and ms > 0
    assert batch.get_option(lq2d.BATCH_THREADS) == threads
    out = batch.solve(1e-10, 2, 2, 5000)
    assert out["status"] == 0 and batch.get_option(lq2d.BATCH_USES_PERSISTENT) == 1
    g = grids[3]
    ref = O.Oracle(O.Problem.from_arrays(g.K, g.N, g.T, g.n, g.m, *g.arrays())).solve(1e-12)
    assert np.linalg.norm(costate_of(probs[3], g, dev) - ref.delta) <= 1e-8 * np.linalg.norm(ref.delta)
    with pytest.raises(lq2d.LQ2DError):
        batch.set_option(lq2d.BATCH_THREADS, 256)
    probs[0].set_precision(1)
    with pytest.raises(lq2d.LQ2DError):
        batch.autotune(2, 2, 1)
    batch.close()


FP32_SCHEDULES = [(32, 4), (64, 4), (64, 2), (128, 2), (32, 2), (64, 1), (32, 0), (64, 0), (128, 0)]
BULK_SHAPES = [(5, 7, 33, 4, 2), (1, 3, 9, 4, 2), (4, 4, 1, 4, 2), (3, 2, 2, 4, 2), (6, 5, 70, 4, 1),
               (2, 9, 4, 4, 2)]


@pytest.mark.parametrize("shape", BULK_SHAPES, ids=["K%dN%dT%d" % s[:3] for s in BULK_SHAPES])
def test_fp32_schedules_match_oracle(dev, shape):
    """Every compiled schedule of the n = 4 FP32 sweeps (bulk-copy kernel with
    1, 2 or 4 time steps per lane at several CTA widths, and the tiled kernel)
    gives the oracle's D_S r (Algorithm 2, S x L sweeps) within the FP32 bound,
    for (S, L) in {(1, 2), (2, 2), (3, 4)}, on odd N, K = 1, T = 1 and 2 and
    ragged tiles; a mixed-precision solve with each schedule reaches the
    oracle's solution."""
    lq2d = lq()
    K, N, T, n, m = shape
    g = synth.random_grid(K, N, T, n, m, seed=900 + 7 * K + 3 * N + T)
    orc = O.Oracle(O.Problem.from_arrays(g.K, g.N, g.T, g.n, g.m, *g.arrays()))
    lam = orc.solve(1e-12).delta
    prob = lq2d.Problem.from_grid(g)
    prob.set_precision(1)
    r = synth.random_vector((g.T + 1, g.nodes, g.n), seed=6)
    rt = torch.from_numpy(r).to(dev)
    refs = {SL: orc.preconditioner(*SL).apply(r.ravel()) for SL in ((1, 2), (2, 2), (3, 4))}
    for thr, steps in FP32_SCHEDULES:
        prob.set_option(lq2d.OPT_SWEEP_THREADS, thr)
        prob.set_option(lq2d.OPT_SWEEP_STEPS, steps)
        st = prob.stats()
        assert (st["sweep_threads"], st["sweep_steps"]) == (thr, steps)
        for SL, ref in refs.items():
            q = torch.empty_like(rt)
            prob.apply_precond_device(SL[0], SL[1], rt, q)
            got = q.cpu().numpy().ravel()
            assert np.isfinite(got).all()
            assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max(), (thr, steps, SL)
        for mode in (1, 2):
            prob.set_precision(mode)
            out = prob.solve(1e-10, 2, 2, 5000)
            assert out["status"] == 0, (thr, steps, mode)
            assert np.linalg.norm(out["costate"] - lam) <= 1e-7 * np.linalg.norm(lam), (thr, steps, mode)
        prob.set_precision(1)
    with pytest.raises(lq2d.LQ2DError):
        prob.set_option(lq2d.OPT_SWEEP_STEPS, 3)
    thr, ms = prob.autotune(2, 2, 2)
    st = prob.stats()
    assert (st["sweep_threads"], st["sweep_steps"]) in FP32_SCHEDULES and thr == st["sweep_threads"]
    prob.close()
