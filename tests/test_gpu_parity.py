"""Parity of the CUDA path against the CPU oracle, through the C-ABI.

Each kernel family is compared element by element with the oracle on the
same seeded inputs: the Delta product (Section II-B), the NBJM
preconditioner (Algorithm 2, Theorem posdef_preconditioner) and the full PCG
solve (Algorithm 1).  Shapes cover several sweep blocks with a ragged tail,
odd N (one-column last pair), single rows and columns, and every compiled
state dimension.  Tolerances: 1e-12 relative for the linear maps (FP64,
different summation order), 1e-8 relative solution error after solving both
sides to 1e-12 (the stated FP64 target).
"""
import json
import os

import numpy as np
import pytest

from oracle import lq2d_oracle as O
from paper_2304_04980_gb300 import synth
from tests import grid_sim

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHAPES = [  # K, N, T, n, m
    (4, 4, 20, 2, 1),
    (9, 7, 33, 4, 2),
    (5, 6, 10, 3, 2),
    (1, 1, 12, 4, 2),
    (3, 5, 9, 1, 1),
    (6, 3, 7, 8, 3),
    (2, 8, 5, 5, 4),
    (7, 2, 4, 6, 1),
    (8, 9, 6, 7, 2),
    (10, 1, 3, 4, 2),
    (1, 10, 2, 2, 2),
    (3, 4, 1, 4, 2),
]
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
    return synth.random_grid(K, N, T, n, m, seed=100 + seed + 7 * K + 3 * N + T + n)


def oracle_for(g):
    return O.Oracle(O.Problem.from_arrays(g.K, g.N, g.T, g.n, g.m, *g.arrays()))


def tdev(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)


def rel_err(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


@pytest.mark.parametrize("shape", SHAPES, ids=IDS)
def test_delta_apply_matches_oracle(dev, shape):
    g = grid_for(shape)
    orc = oracle_for(g)
    prob = lq().Problem.from_grid(g)
    d = synth.random_vector((g.T + 1, g.nodes, g.n), seed=1)
    y = torch.empty_like(tdev(d, dev))
    prob.apply_delta_device(tdev(d, dev), y)
    ref = orc.Delta @ d.ravel()
    got = y.cpu().numpy().ravel()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("S,L", [(1, 2), (2, 2), (3, 4)])
@pytest.mark.parametrize("shape", SHAPES, ids=IDS)
def test_preconditioner_matches_oracle(dev, shape, S, L):
    g = grid_for(shape)
    orc = oracle_for(g)
    prob = lq().Problem.from_grid(g)
    r = synth.random_vector((g.T + 1, g.nodes, g.n), seed=2)
    q = torch.empty_like(tdev(r, dev))
    prob.apply_precond_device(S, L, tdev(r, dev), q)
    ref = orc.preconditioner(S, L).apply(r.ravel())
    got = q.cpu().numpy().ravel()
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("shape", SHAPES, ids=IDS)
def test_solve_matches_oracle(dev, shape):
    g = grid_for(shape)
    orc = oracle_for(g)
    prob = lq().Problem.from_grid(g)
    ref = orc.solve(1e-12, 2, 2, max_iter=5000)
    out = prob.solve(1e-12, 2, 2, 5000)
    assert out["status"] == 0
    assert rel_err(out["costate"], ref.delta) <= 1e-8
    assert rel_err(out["x"], ref.x) <= 1e-8
    assert rel_err(out["u"], ref.u) <= 1e-8
    assert out["rel_kkt"] <= 1e-11
    st = prob.stats()
    assert abs(st["cost"] - ref.cost) <= 1e-9 * abs(ref.cost)
    # iteration counts at a looser tolerance agree up to rounding (reading A18)
    ref10 = orc.solve(1e-10, 2, 2)
    out10 = prob.solve(1e-10, 2, 2, 5000)
    assert abs(out10["iterations"] - ref10.iterations) <= max(2, 0.05 * ref10.iterations)


def test_golden_grid4_T20(dev):
    path = os.path.join(os.path.dirname(__file__), "golden", "grid4_T20.json")
    ref = json.load(open(path))
    g = synth.workload("grid4_T20")
    prob = lq().Problem.from_grid(g)
    out = prob.solve(ref["tol"], ref["S"], ref["L"], 1000)
    assert abs(out["iterations"] - ref["iterations"]) <= 2
    tight = prob.solve(1e-13, 2, 2, 1000)
    assert rel_err(tight["costate"], ref["delta"]) <= 1e-8
    assert rel_err(tight["x"], ref["x"]) <= 1e-8
    assert rel_err(tight["u"], ref["u"]) <= 1e-8
    assert abs(prob.stats()["cost"] - ref["cost"]) <= 1e-10 * ref["cost"]


def test_zero_state_warm_start_and_limits(dev):
    lq2d = lq()
    g = grid_for((5, 4, 8, 4, 2))
    prob = lq2d.Problem.from_grid(g.with_x0(np.zeros_like(g.x0)))
    out = prob.solve(1e-10, 2, 2, 100)
    assert out["iterations"] == 0 and not np.any(out["costate"])
    prob = lq2d.Problem.from_grid(g)
    ref = prob.solve(1e-13, 2, 2, 1000)
    again = prob.solve(1e-10, 2, 2, 1000, delta0=ref["costate"])
    assert again["iterations"] == 0
    capped = prob.solve(1e-12, 2, 2, 3)
    assert capped["status"] == lq2d.ENOCONV and capped["iterations"] == 3
    none = prob.solve(1e-12, 2, 2, 0)
    assert none["status"] == lq2d.ENOCONV and none["iterations"] == 0
    for S, L in ((0, 2), (2, 3), (2, 0)):
        with pytest.raises(lq2d.LQ2DError) as e:
            prob.solve(1e-8, S, L, 10)
        assert e.value.code == lq2d.EINVAL
    with pytest.raises(lq2d.LQ2DError):
        prob.solve(-1.0, 2, 2, 10)


def test_not_positive_definite_and_non_finite_inputs(dev):
    lq2d = lq()
    g = grid_for((3, 3, 4, 2, 1))
    bad = synth.GridLQ(**{**g.__dict__})
    bad.R = g.R.copy()
    bad.R[4] = -bad.R[4]
    with pytest.raises(lq2d.LQ2DError) as e:
        lq2d.Problem.from_grid(bad)
    assert e.value.code == lq2d.ENOTPD
    arrs = [tdev(a, dev) for a in g.arrays()]
    arrs[0][2, 0, 0] = float("nan")
    with pytest.raises(lq2d.LQ2DError) as e:
        lq2d.Problem.from_device(g.K, g.N, g.T, g.n, g.m, *arrs)
    assert e.value.code == lq2d.EINVAL


def test_affine_terms_match_oracle(dev):
    g = grid_for((4, 5, 6, 3, 2))
    w = synth.random_vector((g.T, g.nodes, g.n), seed=9)
    P = O.Problem.from_arrays(g.K, g.N, g.T, g.n, g.m, *g.arrays(), w=w)
    ref = O.Oracle(P).solve(1e-12)
    prob = lq().Problem.from_grid(g)
    prob.set_affine(w)
    out = prob.solve(1e-12, 2, 2, 2000)
    assert rel_err(out["costate"], ref.delta) <= 1e-8
    x_sim = grid_sim.simulate(g.K, g.N, g.T, g.A_self, g.A_nbr, g.B, g.x0, out["u"], w)
    assert rel_err(x_sim, out["x"]) <= 1e-9
    prob.set_affine(None)
    plain = oracle_for(g).solve(1e-12)
    assert rel_err(prob.solve(1e-12, 2, 2, 2000)["costate"], plain.delta) <= 1e-8


def test_infinity_norm_stop_mode(dev):
    lq2d = lq()
    g = grid_for((6, 5, 10, 4, 2))
    orc = oracle_for(g)
    prob = lq2d.Problem.from_grid(g)
    prob.set_option(lq2d.OPT_STOP_MODE, 1)
    out = prob.solve(1e-9, 2, 2, 2000)
    r = orc.r_delta - orc.Delta @ out["costate"].ravel()
    assert np.abs(r).max() < 1e-9
    ref = orc.solve(1e-9, stop="absinf")
    assert abs(out["iterations"] - ref.iterations) <= max(2, 0.05 * ref.iterations)


def test_drivers_agree_and_results_are_deterministic(dev):
    lq2d = lq()
    g = grid_for((9, 7, 33, 4, 2))
    prob = lq2d.Problem.from_grid(g)
    a = prob.solve(1e-10, 2, 2, 1000)
    b = prob.solve(1e-10, 2, 2, 1000)
    prob.set_option(lq2d.OPT_DRIVER, 1)
    c = prob.solve(1e-10, 2, 2, 1000)
    assert a["iterations"] == b["iterations"] == c["iterations"]
    assert np.array_equal(a["costate"], b["costate"]) and np.array_equal(a["costate"], c["costate"])
    prob.set_option(lq2d.OPT_TIMING, 1)
    d = prob.solve(1e-10, 2, 2, 1000)
    st = prob.stats()
    assert np.array_equal(a["costate"], d["costate"])
    assert st["sweep_launches"] == (d["iterations"] - 1) * 4 + 1
    assert st["delta_launches"] == d["iterations"] and st["sweep_ms"] > 0


def test_device_entry_points_and_update(dev):
    lq2d = lq()
    g = grid_for((6, 6, 12, 4, 2))
    g2 = grid_for((6, 6, 12, 4, 2), seed=5)
    arrs = [tdev(a, dev) for a in g.arrays()]
    prob = lq2d.Problem.from_device(g.K, g.N, g.T, g.n, g.m, *arrs)
    x = torch.empty((g.T + 1, g.nodes, g.n), dtype=torch.float64, device=dev)
    u = torch.empty((g.T, g.nodes, g.m), dtype=torch.float64, device=dev)
    lam = torch.empty_like(x)
    prob.solve_device(1e-12, 2, 2, 1000, x=x, u=u, costate=lam)
    assert rel_err(lam.cpu().numpy(), oracle_for(g).solve(1e-12).delta) <= 1e-8
    prob.update_device(*[tdev(a, dev) for a in g2.arrays()])
    prob.solve_device(1e-12, 2, 2, 1000, x=x, u=u, costate=lam)
    ref2 = oracle_for(g2).solve(1e-12)
    assert rel_err(lam.cpu().numpy(), ref2.delta) <= 1e-8
    assert rel_err(u.cpu().numpy(), ref2.u) <= 1e-8


# --------------------------------------------------------------------------
# full-size workload (K = N = 64, T = 100): sampled rows and properties
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def big(dev):
    g = synth.workload("grid64_T100")
    prob = lq().Problem.from_grid(g)
    return g, prob


def test_full_size_delta_rows(dev, big):
    g, prob = big
    d = synth.random_vector((g.T + 1, g.nodes, g.n), seed=3)
    y = torch.empty_like(tdev(d, dev))
    prob.apply_delta_device(tdev(d, dev), y)
    P = O.Problem.from_arrays(g.K, g.N, g.T, g.n, g.m, *g.arrays())
    rows = np.random.default_rng(4).choice(P.dim_x, 64, replace=False)
    rows = np.concatenate([rows, [0, P.dim_x - 1, g.nodes * g.n - 1, g.nodes * g.n]])
    ref = O.delta_rows_matrix_free(P, rows, d.ravel())
    got = y.cpu().numpy().ravel()[rows]
    assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


def test_full_size_preconditioner_is_symmetric_positive(dev, big):
    g, prob = big
    a = synth.random_vector((g.T + 1, g.nodes, g.n), seed=5)
    b = synth.random_vector((g.T + 1, g.nodes, g.n), seed=6)
    pa = torch.empty_like(tdev(a, dev))
    pb = torch.empty_like(pa)
    prob.apply_precond_device(2, 2, tdev(a, dev), pa)
    prob.apply_precond_device(2, 2, tdev(b, dev), pb)
    pa, pb = pa.cpu().numpy().ravel(), pb.cpu().numpy().ravel()
    assert abs(a.ravel() @ pb - b.ravel() @ pa) <= 1e-10 * abs(a.ravel() @ pa)
    assert a.ravel() @ pa > 0 and b.ravel() @ pb > 0


def test_full_size_solve_properties(dev, big):
    g, prob = big
    out = prob.solve(1e-10, 2, 2, 5000)
    assert out["status"] == 0 and out["rel_kkt"] <= 1e-10
    # every step of (x, u) satisfies the dynamics (checked one step at a
    # time: the open-loop dynamics of this workload are unstable, so a
    # forward simulation would amplify the 1e-10 residual)
    step_res = [out["x"][0] - g.x0] + [
        out["x"][t + 1] - grid_sim.step(g.K, g.N, g.A_self, g.A_nbr, g.B, out["x"][t], out["u"][t])
        for t in range(g.T)]
    assert np.linalg.norm(np.array(step_res)) <= 1e-9 * np.linalg.norm(g.x0)
    # terminal costate: delta_T = -Q_T x_T (reading A3)
    lamT = -np.einsum("pab,pb->pa", g.Q_T, out["x"][-1])
    assert rel_err(out["costate"][-1], lamT) <= 1e-12
    # cost from states and inputs equals 1/2 delta' r_delta
    J = grid_sim.cost(g.Q, g.R, g.Q_T, out["x"], out["u"])
    half = -0.5 * float(out["costate"][0].ravel() @ g.x0.ravel())
    assert abs(J - half) <= 1e-7 * J
    assert abs(prob.stats()["cost"] - J) <= 1e-9 * J
    # sampled rows of the true residual, from the oracle's row evaluation
    P = O.Problem.from_arrays(g.K, g.N, g.T, g.n, g.m, *g.arrays())
    rows = np.random.default_rng(7).choice(P.dim_x, 48, replace=False)
    rd = np.zeros(P.dim_x)
    rd[: g.nodes * g.n] = -g.x0.ravel()
    res = rd[rows] - O.delta_rows_matrix_free(P, rows, out["costate"].ravel())
    assert np.abs(res).max() <= 1e-9 * np.linalg.norm(rd)


def test_full_size_solution_matches_oracle(dev, big):
    """The whole K = N = 64, T = 100 solve against the oracle's PCG, both run
    to 1e-11: relative solution error within the FP64 target 1e-8."""
    g, prob = big
    orc = oracle_for(g)
    ref = orc.solve(1e-11, 2, 2, max_iter=2000)
    out = prob.solve(1e-11, 2, 2, 2000)
    assert ref.converged and out["status"] == 0
    assert rel_err(out["costate"], ref.delta) <= 1e-8
    assert rel_err(out["x"], ref.x) <= 1e-8
    assert rel_err(out["u"], ref.u) <= 1e-8
    assert abs(out["iterations"] - ref.iterations) <= max(2, 0.05 * ref.iterations)
