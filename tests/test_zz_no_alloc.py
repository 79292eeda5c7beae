"""The allocation-free Delta product (lq2d_apply_delta_static), through the
C-ABI, against the handle-based one (lq2d_apply_delta_device) and against the
oracle's Delta = A~ Q~^-1 A~' + B~ R~^-1 B~' (Section II-B).

The allocation-free form exists for callers that may not allocate device
memory while they run: fixed-period control loops, where an allocator call
adds latency they cannot bound, and host frameworks that own every device
allocation.  Its scratch is one fixed array in the library.  Two calls in a
row on different problems check that the shared scratch, which keeps the
previous call's contents, does not leak into the next result; the free
device memory is read around further calls to check that they allocate
nothing.  This file is collected last so that a failure here stops a -x run
only after every other test has run."""
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


SHAPES = [(9, 7, 33, 4, 2), (6, 5, 12, 3, 2), (9, 7, 33, 4, 2)]


def test_static_scratch_delta_matches_handle_entry_point(dev):
    from paper_2304_04980_gb300 import lq2d
    for call, (K, N, T, n, m) in enumerate(SHAPES):
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


def test_static_scratch_delta_matches_oracle(dev):
    """Element by element against the oracle's assembled Delta times d, on
    two calls in a row (odd N, K = 1, n = 1 included)."""
    from oracle import lq2d_oracle as O
    from paper_2304_04980_gb300 import lq2d
    for call, (K, N, T, n, m) in enumerate([(5, 7, 9, 4, 2), (1, 3, 6, 1, 1), (4, 4, 20, 2, 1)]):
        g = synth.random_grid(K, N, T, n, m, seed=700 + call)
        d = synth.random_vector((T + 1, K * N, n), seed=800 + call)
        orc = O.Oracle(O.Problem.from_arrays(K, N, T, n, m, *g.arrays()))
        want = (orc.Delta @ d.ravel()).reshape(d.shape)
        out = torch.full(d.shape, float("nan"), dtype=torch.float64, device=dev)
        lq2d.apply_delta_static(K, N, T, n, m, *[tdev(a, dev) for a in g.arrays()[:6]], tdev(d, dev), out)
        got = out.cpu().numpy()
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_static_scratch_calls_allocate_no_device_memory(dev):
    from paper_2304_04980_gb300 import lq2d
    K, N, T, n, m = SHAPES[0]
    args = []
    for s, (K, N, T, n, m) in enumerate(SHAPES[:2]):
        g = synth.random_grid(K, N, T, n, m, seed=900 + s)
        din = tdev(synth.random_vector((T + 1, K * N, n), seed=950 + s), dev)
        args.append(((K, N, T, n, m), [tdev(a, dev) for a in g.arrays()[:6]], din, torch.empty_like(din)))
    # warm-up: the first call loads the module and looks up the array
    for shape, blocks, din, out in args:
        lq2d.apply_delta_static(*shape, *blocks, din, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(dev)
    for _ in range(3):
        for shape, blocks, din, out in args:
            lq2d.apply_delta_static(*shape, *blocks, din, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(dev)
    assert free1 == free0


def test_static_scratch_reports_a_non_spd_weight(dev):
    """Q with a negative eigenvalue is a host-visible status, not a fault;
    the next call with valid data still matches the handle's product."""
    from paper_2304_04980_gb300 import lq2d
    K, N, T, n, m = 3, 4, 5, 2, 1
    g = synth.random_grid(K, N, T, n, m, seed=31)
    Q = g.Q.copy()
    Q[5] = np.diag([1.0, -2.0])
    blocks = [tdev(a, dev) for a in g.arrays()[:6]]
    bad = list(blocks)
    bad[3] = tdev(Q, dev)
    din = tdev(synth.random_vector((T + 1, K * N, n), seed=32), dev)
    out = torch.empty_like(din)
    with pytest.raises(lq2d.LQ2DError) as e:
        lq2d.apply_delta_static(K, N, T, n, m, *bad, din, out)
    assert e.value.code == lq2d.ENOTPD
    lq2d.apply_delta_static(K, N, T, n, m, *blocks, din, out)
    ref = torch.empty_like(din)
    with lq2d.Problem.from_grid(g) as prob:
        prob.apply_delta_device(din, ref)
    assert torch.abs(out - ref).max().item() <= 1e-12 * torch.abs(ref).max().item()


def test_static_scratch_rejects_sizes_beyond_its_array_and_overlap(dev):
    from paper_2304_04980_gb300 import lq2d
    K, N, T, n, m = 128, 128, 100, 4, 2
    tiny = torch.zeros(8, dtype=torch.float64, device=dev)
    with pytest.raises(lq2d.LQ2DError) as e:
        lq2d.apply_delta_static(K, N, T, n, m, *([tiny] * 6), tiny, tiny)
    assert e.value.code == lq2d.EINVAL and "scratch" in str(e.value)
    K, N, T, n, m = 2, 2, 3, 2, 1
    g = synth.random_grid(K, N, T, n, m, seed=41)
    blocks = [tdev(a, dev) for a in g.arrays()[:6]]
    buf = torch.zeros(2 * (T + 1) * K * N * n, dtype=torch.float64, device=dev)
    with pytest.raises(lq2d.LQ2DError) as e:
        lq2d.apply_delta_static(K, N, T, n, m, *blocks, buf, buf[3:])
    assert e.value.code == lq2d.EINVAL and "overlap" in str(e.value)
