"""The allocation-free Delta product (lq2d_apply_delta_static) against the
handle-based one (lq2d_apply_delta_device), through the C-ABI.

The allocation-free form exists for callers that may not allocate device
memory while they run (fixed-period control loops, host frameworks that own
all device allocations); its scratch is one fixed array in the library.  Two
calls in a row on different problems check that the shared scratch, which
keeps the previous call's contents, does not leak into the next result.
This file is collected last so that a failure here stops a -x run only
after every other test has run."""
import numpy as np
import pytest

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


def tdev(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev)


def test_static_scratch_delta_matches_handle_entry_point(dev):
    from paper_2304_04980_gb300 import lq2d
    shapes = [(9, 7, 33, 4, 2), (6, 5, 12, 3, 2), (9, 7, 33, 4, 2)]
    for call, (K, N, T, n, m) in enumerate(shapes):
        g = synth.random_grid(K, N, T, n, m, seed=500 + call)
        d = synth.random_vector((T + 1, K * N, n), seed=600 + call)
        blocks = [tdev(a, dev) for a in g.arrays()[:6]]
        din = tdev(d, dev)
        ref = torch.empty_like(din)
        with lq2d.Problem.from_grid(g) as prob:
            prob.apply_delta_device(din, ref)
        out = torch.full_like(din, float("nan"))
        lq2d.apply_delta_static(K, N, T, n, m, *blocks, din, out)
        ref_np, out_np = ref.cpu().numpy(), out.cpu().numpy()
        assert np.isfinite(out_np).all()
        assert np.abs(out_np - ref_np).max() <= 1e-12 * np.abs(ref_np).max()


def test_static_scratch_rejects_sizes_beyond_its_array(dev):
    from paper_2304_04980_gb300 import lq2d
    K, N, T, n, m = 128, 128, 100, 4, 2
    tiny = torch.zeros(8, dtype=torch.float64, device=dev)
    with pytest.raises(lq2d.LQ2DError) as e:
        lq2d.apply_delta_static(K, N, T, n, m, *([tiny] * 6), tiny, tiny)
    assert e.value.code == lq2d.EINVAL and "scratch" in str(e.value)
