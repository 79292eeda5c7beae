"""Mixed precision (FP32 preconditioner, FP64 residual, dots and updates)
against the FP64 oracle, through the C-ABI.

The FP32 sweeps change only the preconditioner; the tolerance still applies
to the FP64 residual, so the solution must match the oracle to the stated
mixed-precision bound (relative error <= 1e-6) and, in practice, far better.
For the preconditioner alone the bound is FP32 rounding (unit roundoff
6e-8) amplified by the conditioning of the Phi_bar blocks and the S x L
sweeps: 1e-4 relative to the largest entry.
"""
import numpy as np
import pytest

from oracle import lq2d_oracle as O
from paper_2304_04980_gb300 import synth
from tests import grid_sim

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHAPES = [(4, 4, 20, 2, 1), (9, 7, 33, 4, 2), (5, 6, 10, 3, 2), (3, 5, 9, 1, 1), (6, 3, 7, 8, 3)]
IDS = ["K%dN%dT%dn%dm%d" % s for s in SHAPES]


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
    return synth.random_grid(K, N, T, n, m, seed=200 + seed + 7 * K + 3 * N + T + n)


def oracle_for(g):
    return O.Oracle(O.Problem.from_arrays(g.K, g.N, g.T, g.n, g.m, *g.arrays()))


def tdev(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)


def rel_err(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


@pytest.mark.parametrize("shape", SHAPES, ids=IDS)
def test_fp32_preconditioner_matches_oracle(dev, shape):
    g = grid_for(shape)
    prob = lq().Problem.from_grid(g)
    prob.set_precision(1)
    r = synth.random_vector((g.T + 1, g.nodes, g.n), seed=3)
    q = torch.empty_like(tdev(r, dev))
    prob.apply_precond_device(2, 2, tdev(r, dev), q)
    ref = oracle_for(g).preconditioner(2, 2).apply(r.ravel())
    got = q.cpu().numpy().ravel()
    assert np.abs(got - ref).max() <= 1e-4 * np.abs(ref).max()
    # and it is not the FP64 result: the FP32 path really ran
    prob.set_precision(0)
    q64 = torch.empty_like(q)
    prob.apply_precond_device(2, 2, tdev(r, dev), q64)
    assert not torch.equal(q, q64)


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("shape", SHAPES, ids=IDS)
def test_mixed_solve_matches_oracle(dev, shape, mode):
    g = grid_for(shape)
    orc = oracle_for(g)
    ref = orc.solve(1e-12, 2, 2, max_iter=5000)
    prob = lq().Problem.from_grid(g)
    plain = prob.solve(1e-10, 2, 2, 5000)
    prob.set_precision(mode)
    out = prob.solve(1e-10, 2, 2, 5000)
    assert out["status"] == 0 and out["rel_kkt"] <= 1e-10
    for key, refv in (("costate", ref.delta), ("x", ref.x), ("u", ref.u)):
        assert rel_err(out[key], refv) <= 1e-6
    if mode == 1:
        # FP32 rounding inside the preconditioner costs at most a few iterations
        assert out["iterations"] <= int(1.25 * plain["iterations"]) + 3
    else:
        # the FP32 product's residual is replaced by the FP64 one once per
        # drop of 1e4, keeping the direction: no restart, few extra steps
        st = prob.stats()
        assert st["residual_replacements"] >= 1
        assert out["iterations"] <= int(1.5 * plain["iterations"]) + 5


def test_mode_switch_and_update_refresh_fp32_operands(dev):
    lq2d = lq()
    g1 = grid_for((6, 6, 12, 4, 2))
    g2 = grid_for((6, 6, 12, 4, 2), seed=5)
    prob = lq2d.Problem.from_device(g1.K, g1.N, g1.T, g1.n, g1.m, *[tdev(a, dev) for a in g1.arrays()])
    prob.set_precision(1)
    a = prob.solve(1e-11, 2, 2, 2000)
    prob.update_device(*[tdev(a_, dev) for a_ in g2.arrays()])
    b = prob.solve(1e-11, 2, 2, 2000)
    assert rel_err(b["costate"], oracle_for(g2).solve(1e-12).delta) <= 1e-6
    prob.set_precision(0)
    c = prob.solve(1e-11, 2, 2, 2000)
    assert rel_err(b["costate"], c["costate"]) <= 1e-6
    prob.set_precision(1)
    d = prob.solve(1e-11, 2, 2, 2000)
    assert np.array_equal(b["costate"], d["costate"])
    assert rel_err(a["costate"], oracle_for(g1).solve(1e-12).delta) <= 1e-6
    with pytest.raises(lq2d.LQ2DError):
        prob.set_precision(3)


@pytest.mark.parametrize("mode", [1, 2])
def test_mixed_full_size_bench_workload(dev, mode):
    """K = N = 64, T = 100: mixed and FP64 solutions agree, the mixed one
    satisfies the dynamics step by step, and both pass the true residual."""
    g = synth.workload("grid64_T100")
    prob = lq().Problem.from_grid(g)
    plain = prob.solve(1e-10, 2, 2, 5000)
    prob.set_precision(mode)
    out = prob.solve(1e-10, 2, 2, 5000)
    assert out["status"] == 0 and out["rel_kkt"] <= 1e-10
    assert rel_err(out["costate"], plain["costate"]) <= 1e-6
    res = [out["x"][0] - g.x0] + [
        out["x"][t + 1] - grid_sim.step(g.K, g.N, g.A_self, g.A_nbr, g.B, out["x"][t], out["u"][t])
        for t in range(g.T)]
    assert np.linalg.norm(np.array(res)) <= 1e-9 * np.linalg.norm(g.x0)
