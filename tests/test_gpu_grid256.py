"""The K = N = 256, T = 200 grid (52.7 M multipliers) solved through the C-ABI
in each precision mode, checked over every row against the oracle's slab-by-
slab evaluation of the definitions of Section II-B:

* the relative true residual ||r_delta - Delta delta||_2 / ||r_delta||_2 of
  the returned multipliers, with Delta = A~ Q~^-1 A~' + B~ R~^-1 B~' applied
  one time slab at a time (the solve's own stop test is confirmed on its
  own true residual; this recomputes it independently of the CUDA path);
* x = Q~^-1 A~' delta and u = R~^-1 B~' delta against the returned x, u;
* the mixed-precision multipliers against the FP64 ones (relative error
  <= 1e-6, the mixed-precision bound).
The tolerance is the bench's 1e-8; the oracle's residual may differ from the
solver's by rounding of the product only (about 1e-15 relative), so the
test allows 1e-8 (1 + 1e-6).
"""
import numpy as np
import pytest

from oracle import lq2d_oracle as O
from paper_2304_04980_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-8


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2304_04980_gb300 import build
    build.build()
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def case(dev):
    from paper_2304_04980_gb300 import lq2d
    g = synth.workload("grid256_T200")
    P = O.Problem.from_arrays(g.K, g.N, g.T, g.n, g.m, *g.arrays())
    blocks = O.slab_blocks(P)
    prob = lq2d.Problem.from_grid(g)
    results = {}
    yield g, P, blocks, prob, results
    prob.close()


def rel_err(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_grid256_true_residual_and_recovery_over_every_row(case, mode):
    g, P, blocks, prob, results = case
    prob.set_precision(mode)
    out = prob.solve(TOL, 2, 2, 5000)
    assert out["status"] == 0 and out["rel_kkt"] <= TOL
    delta = out["costate"]
    res = O.true_residual_slabs(P, delta, blocks)
    assert res <= TOL * (1 + 1e-6), res
    # the solver's reported KKT residual is the same quantity up to rounding
    assert abs(res - out["rel_kkt"]) <= 1e-12
    x, u = O.recover_slabs(P, delta, blocks)
    assert rel_err(out["x"], x) <= 1e-13
    assert rel_err(out["u"], u) <= 1e-13
    results[mode] = delta
    if mode > 0 and 0 in results:
        assert rel_err(delta, results[0]) <= 1e-6
