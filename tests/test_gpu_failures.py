"""Failure detection through the C-ABI without any GPU fault: a non-finite
warm start or initial state makes the residual non-finite, the device
state records a breakdown, the call returns LQ2D_EBREAKDOWN, and the
handle stays usable (the next solve is correct).  Iteration caps return
LQ2D_ENOCONV with the outputs written."""
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


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_non_finite_warm_start_is_a_breakdown_and_the_handle_recovers(dev, mode):
    lq2d = lq()
    g = synth.random_grid(5, 4, 9, 4, 2, seed=31)
    prob = lq2d.Problem.from_grid(g)
    prob.set_precision(mode)
    bad = np.zeros((g.T + 1, g.nodes, g.n))
    bad[3, 7, 1] = np.nan
    with pytest.raises(lq2d.LQ2DError) as e:
        prob.solve(1e-10, 2, 2, 500, delta0=bad, allow=())
    assert e.value.code == lq2d.EBREAKDOWN
    out = prob.solve(1e-10, 2, 2, 500)
    ref = O.Oracle(O.Problem.from_arrays(g.K, g.N, g.T, g.n, g.m, *g.arrays())).solve(1e-12)
    assert out["status"] == 0
    assert np.linalg.norm(out["costate"] - ref.delta) <= 1e-7 * np.linalg.norm(ref.delta)
    prob.close()


def test_non_finite_initial_state_in_a_multi_rhs_solve(dev):
    lq2d = lq()
    g = synth.random_grid(5, 4, 9, 4, 2, seed=32)
    prob = lq2d.Problem.from_grid(g)
    x0s = np.random.default_rng(1).standard_normal((4, g.nodes, g.n))
    x0s[2, 3, 0] = np.inf
    with pytest.raises(lq2d.LQ2DError) as e:
        prob.solve_multi_device(4, torch.from_numpy(x0s).to(dev), 1e-10, 2, 2, 500, allow=())
    assert e.value.code == lq2d.EBREAKDOWN
    x0s[2, 3, 0] = 0.5
    lam = torch.empty((4, g.T + 1, g.nodes, g.n), dtype=torch.float64, device=dev)
    out = prob.solve_multi_device(4, torch.from_numpy(x0s).to(dev), 1e-10, 2, 2, 500, costate=lam)
    assert out["status"] == 0
    ref = O.Oracle(O.Problem.from_arrays(g.K, g.N, g.T, g.n, g.m, *g.with_x0(x0s[2]).arrays())).solve(1e-12)
    assert np.linalg.norm(lam[2].cpu().numpy() - ref.delta) <= 1e-7 * np.linalg.norm(ref.delta)
    prob.close()


def test_iteration_cap_returns_enoconv_with_outputs(dev):
    lq2d = lq()
    g = synth.random_grid(6, 6, 12, 4, 2, seed=33)
    prob = lq2d.Problem.from_grid(g)
    out = prob.solve(1e-14, 2, 2, 3)
    assert out["status"] == lq2d.ENOCONV and out["iterations"] == 3
    assert np.all(np.isfinite(out["costate"])) and np.abs(out["costate"]).max() > 0
    # the batch reports it per problem
    batch = lq2d.Batch([prob])
    res = batch.solve(1e-14, 2, 2, 3)
    assert res["statuses"][0] == lq2d.ENOCONV
    batch.close()
    prob.close()


@pytest.mark.parametrize("k", [1, 2, 16, 24])
def test_allocation_failure_returns_enomem_and_releases_memory(dev, k, monkeypatch):
    """A device allocation that fails during creation (injected on the host
    through LQ2D_FAIL_ALLOC_AT, no GPU memory exhausted) returns
    LQ2D_ENOMEM, releases the allocations made before it, and leaves the
    library usable."""
    lq2d = lq()
    g = synth.workload("grid64_T100")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(dev)
    monkeypatch.setenv("LQ2D_FAIL_ALLOC_AT", str(k))
    with pytest.raises(lq2d.LQ2DError) as e:
        lq2d.Problem.from_grid(g)
    assert e.value.code == lq2d.ENOMEM and "cudaMalloc" in str(e.value)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(dev)
    # the allocations before the k-th hold over 100 MB at k = 24
    assert abs(free1 - free0) <= 8 << 20
    monkeypatch.delenv("LQ2D_FAIL_ALLOC_AT")
    small = synth.random_grid(3, 3, 5, 2, 1, seed=3)
    with lq2d.Problem.from_grid(small) as prob:
        out = prob.solve(1e-10, 2, 2, 200)
    assert out["status"] == 0
