"""The warm-start network's CUDA kernels against the CPU oracle (forward
pass, loss, gradients, Adam step), and what the trained network gains:
fewer PCG iterations from its guess than from zero, to the same solution."""
import numpy as np
import pytest

from oracle import lq2d_oracle as O
from oracle import warmstart_net as W
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


# (K, N, T, n, channels, layers, batch): ragged tiles of the 64 x 64 GEMM
# tiles in every dimension, a one-row grid, a linear (one-layer) net
NETS = [(5, 6, 3, 2, 8, 3, 2), (9, 13, 2, 4, 16, 2, 3), (1, 7, 4, 1, 5, 2, 1), (4, 4, 1, 3, 6, 1, 2),
        (12, 11, 8, 4, 70, 3, 2)]
IDS = ["K%dN%dT%dn%dc%dl%db%d" % s for s in NETS]


def setup_net(shape, seed=0):
    K, N, T, n, ch, layers, batch = shape
    lq2d = lq()
    net = lq2d.WarmStartNet(K, N, T, n, ch, layers, batch, sigma=1.7)
    params = synth.warmstart_init(net.layer_sizes(), seed, out_scale=1.0)
    # non-zero biases so that the bias paths are exercised
    r = np.random.default_rng(seed + 1)
    flat = params.copy()
    off = 0
    for ci, co in zip(net.layer_sizes()[:-1], net.layer_sizes()[1:]):
        off += co * ci * 9
        flat[off:off + co] = (r.standard_normal(co) * 0.1).astype(np.float32)
        off += co
    net.set_params(flat)
    x0 = r.standard_normal((batch, K * N, n))
    c = r.uniform(0.02, 0.2, size=batch)
    tgt = r.standard_normal((batch, T + 1, K * N, n))
    return net, flat, x0, c, tgt


def oracle_params(net, flat):
    """The weights as the forward pass uses them (bfloat16), FP32 biases."""
    return [(W.bf16_round(w), b.astype(np.float64)) for w, b in net.unflatten(flat)]


def oracle_inputs(net, x0, c):
    return np.stack([W.features(x0[b], c[b], net.K, net.N, net.n) for b in range(len(c))])


@pytest.mark.parametrize("shape", NETS, ids=IDS)
def test_forward_matches_oracle(dev, shape):
    net, flat, x0, c, _ = setup_net(shape)
    batch = shape[-1]
    out = torch.empty((batch, net.T + 1, net.K * net.N, net.n), dtype=torch.float64, device=dev)
    net.forward_device(batch, torch.from_numpy(x0).to(dev), c, out)
    yhat, _ = W.forward(oracle_params(net, flat), oracle_inputs(net, x0, c))
    ref = np.stack([W.to_delta(yhat[b], net.K, net.N, net.T, net.n, net.sigma) for b in range(batch)])
    got = out.cpu().numpy()
    assert np.abs(got - ref).max() <= 2e-5 * np.abs(ref).max()
    net.close()


@pytest.mark.parametrize("shape", NETS, ids=IDS)
def test_loss_and_gradients_match_oracle(dev, shape):
    net, flat, x0, c, tgt = setup_net(shape, seed=3)
    batch = shape[-1]
    loss, g = net.loss_grad_device(batch, torch.from_numpy(x0).to(dev), c, torch.from_numpy(tgt).to(dev))
    scaled = np.stack([W.from_delta(tgt[b], net.K, net.N, net.T, net.n, net.sigma) for b in range(batch)])
    ref_loss, ref_grads = W.loss_and_grads(oracle_params(net, flat), oracle_inputs(net, x0, c), scaled)
    assert abs(loss - ref_loss) <= 1e-5 * ref_loss
    for (gw, gb), (rw, rb) in zip(net.unflatten(g), ref_grads):
        assert np.abs(gw - rw).max() <= 1e-4 * max(np.abs(rw).max(), 1e-30)
        assert np.abs(gb - rb).max() <= 1e-4 * max(np.abs(rb).max(), 1e-30)
    # the call leaves the parameters alone
    assert np.array_equal(net.get_params(), flat)
    net.close()


def test_adam_step_matches_oracle(dev):
    shape = NETS[0]
    net, flat, x0, c, tgt = setup_net(shape, seed=5)
    batch = shape[-1]
    xd, td = torch.from_numpy(x0).to(dev), torch.from_numpy(tgt).to(dev)
    _, g = net.loss_grad_device(batch, xd, c, td)
    lr = 3e-3
    net.train_step_device(batch, xd, c, td, lr)
    p1 = net.get_params().astype(np.float64)
    ref, m, v = W.adam_step(flat.astype(np.float64), g.astype(np.float64), np.zeros(flat.size), np.zeros(flat.size),
                            1, lr)
    assert np.abs(p1 - ref).max() <= 1e-3 * lr
    # second step: moments carried over
    _, g2 = net.loss_grad_device(batch, xd, c, td)
    net.train_step_device(batch, xd, c, td, lr)
    ref2, _, _ = W.adam_step(ref, g2.astype(np.float64), m, v, 2, lr)
    assert np.abs(net.get_params() - ref2).max() <= 2e-3 * lr
    net.close()


def test_bad_batch_is_rejected(dev):
    lq2d = lq()
    net = lq2d.WarmStartNet(4, 4, 2, 2, 4, 2, 2)
    x = torch.zeros((3, 16, 2), dtype=torch.float64, device=dev)
    out = torch.empty((3, 3, 16, 2), dtype=torch.float64, device=dev)
    with pytest.raises(lq2d.LQ2DError):
        net.forward_device(3, x, [0.1, 0.1, 0.1], out)
    net.close()


def test_any_initial_iterate_reaches_the_same_solution(dev):
    """Algorithm 1 from a poor delta^(0) (random) and from zero converge to
    the same costates, matching the oracle."""
    lq2d = lq()
    fam = synth.warmstart_family(6, 5, 7, 2, 1, seed=9)
    g = fam.instance(1001)
    prob = lq2d.Problem.from_grid(g)
    zero = prob.solve(1e-11, 2, 2, 5000)
    bad = prob.solve(1e-11, 2, 2, 5000, delta0=synth.random_vector((g.T + 1, g.nodes, g.n), seed=4) * 10)
    ref = O.Oracle(O.Problem.from_arrays(g.K, g.N, g.T, g.n, g.m, *g.arrays())).solve(1e-12).delta
    for out in (zero, bad):
        assert out["status"] == 0
        assert np.linalg.norm(out["costate"] - ref) <= 1e-8 * np.linalg.norm(ref)
    # the exact solution as the start: no iterations needed
    exact = prob.solve(1e-8, 2, 2, 5000, delta0=zero["costate"])
    assert exact["iterations"] <= 1


def test_trained_network_reduces_iterations(dev):
    """Train on solver outputs of a 16 x 16, T = 20 family, then solve
    held-out instances from the network's guess and from zero."""
    from paper_2304_04980_gb300 import warmstart
    fam = synth.warmstart_family(16, 16, 20, 4, 2, seed=11)
    ws = warmstart.WarmStart(fam, channels=32, layers=4, batch=8, seed=0)
    ws.generate(range(1000, 1064), tol=1e-8, precision=0)
    sigma = float(ws.targets.std())
    ws.net.close()
    ws.net = lq().WarmStartNet(fam.K, fam.N, fam.T, fam.n, 32, 4, 8, sigma)
    ws.net.set_params(synth.warmstart_init(ws.net.layer_sizes(), 0, 0.1))
    losses = ws.fit(400, lr=2e-3, lr_final=2e-4)
    assert losses[-20:].mean() < 0.5 * losses[:5].mean()
    zero_its, warm_its = [], []
    for seed in range(5000, 5010):
        z = ws.solve(seed, tol=1e-8, warm=False)
        w = ws.solve(seed, tol=1e-8, warm=True)
        assert z["status"] == 0 and w["status"] == 0
        diff = torch.linalg.norm(w["costate"] - z["costate"]) / torch.linalg.norm(z["costate"])
        assert float(diff) <= 1e-6
        zero_its.append(z["iterations"])
        warm_its.append(w["iterations"])
    assert np.mean(warm_its) < np.mean(zero_its)
    ws.close()


def test_grouped_generation_matches_the_oracle(dev):
    """Training pairs from multi-right-hand-side solves: groups of 16
    consecutive seeds (the last one ragged) share the coupling of the group's
    first seed, each pair keeps its own x0, and every target is that
    instance's costate."""
    from paper_2304_04980_gb300 import warmstart
    fam = synth.warmstart_family(8, 6, 9, 4, 2, seed=12)
    ws = warmstart.WarmStart(fam, channels=8, layers=2, batch=4, seed=0)
    seeds = list(range(2000, 2040))
    ws.generate_grouped(seeds, tol=1e-10, group=16)
    for k in (0, 15, 16, 31, 39):
        c = fam.instance_params(seeds[k - k % 16])[0]
        x0 = fam.instance_params(seeds[k])[1]
        assert ws.couplings[k] == c
        assert np.array_equal(ws.x0[k].cpu().numpy(), x0)
        g = fam.grid(c, x0)
        ref = O.Oracle(O.Problem.from_arrays(g.K, g.N, g.T, g.n, g.m, *g.arrays())).solve(1e-12).delta
        got = ws.targets[k].cpu().numpy()
        assert np.linalg.norm(got - ref) <= 1e-7 * np.linalg.norm(ref)
    assert np.all(ws.iterations > 0)
    ws.close()


def test_online_training_keeps_a_ring_buffer_of_solved_pairs(dev):
    """fit_online: five groups of 8 seeds through a buffer of 16 pairs, three
    Adam steps after each group; the buffer ends holding the last two
    groups, each target that instance's costate."""
    from paper_2304_04980_gb300 import warmstart
    fam = synth.warmstart_family(6, 6, 7, 4, 2, seed=13)
    ws = warmstart.WarmStart(fam, channels=8, layers=2, batch=4, seed=0)
    seeds = list(range(3000, 3040))
    losses, gen_s, train_s, count = ws.fit_online(seeds, 3, tol=1e-10, group=8, buffer=16, lr=1e-3,
                                                  lr_final=1e-4)
    assert count == 40 and len(losses) == 15 and np.all(np.isfinite(losses))
    assert gen_s > 0 and train_s > 0 and len(ws.iterations) == 40
    # slot 0..7: group 4 (seeds 3032..3039), slot 8..15: group 3 (3024..3031)
    for slot, sd, first in ((0, 3032, 3032), (7, 3039, 3032), (8, 3024, 3024), (15, 3031, 3024)):
        c = fam.instance_params(first)[0]
        x0 = fam.instance_params(sd)[1]
        assert ws.couplings[slot] == c
        assert np.array_equal(ws.x0[slot].cpu().numpy(), x0)
        g = fam.grid(c, x0)
        ref = O.Oracle(O.Problem.from_arrays(g.K, g.N, g.T, g.n, g.m, *g.arrays())).solve(1e-12).delta
        assert np.linalg.norm(ws.targets[slot].cpu().numpy() - ref) <= 1e-7 * np.linalg.norm(ref)
    with pytest.raises(ValueError):
        ws.fit_online(seeds, 1, group=8, buffer=12)
    ws.close()


def test_network_of_the_full_architecture_reduces_iterations_on_128x128x100(dev):
    """The learned warm start at its own size: 6 layers of 3 x 3 convolutions
    with 64 channels on the K = N = 128, n = 4, m = 2, T = 100 family,
    trained on 256 solver-generated pairs (grouped multi-right-hand-side
    solves, a reduced training set), then held-out instances solved from the
    network's guess and from zero in FP64: fewer PCG steps from the guess,
    and the same costate within 1e-6 (Algorithm 1 accepts any delta^(0))."""
    from paper_2304_04980_gb300 import warmstart
    fam = synth.warmstart_family()
    assert (fam.K, fam.N, fam.T, fam.n, fam.m) == (128, 128, 100, 4, 2)
    ws = warmstart.WarmStart(fam, channels=64, layers=6, batch=8, seed=0)
    ws.generate_grouped(range(1000, 1256), tol=1e-6, group=32)
    sigma = float(ws.targets.std())
    ws.net.close()
    ws.net = lq().WarmStartNet(fam.K, fam.N, fam.T, fam.n, 64, 6, 8, sigma)
    ws.net.set_params(synth.warmstart_init(ws.net.layer_sizes(), 0, 0.1))
    losses = ws.fit(800, lr=1e-3, lr_final=5e-5)
    assert losses[-50:].mean() < 0.2 * losses[:10].mean()
    zero_its, warm_its = [], []
    for seed in range(100000, 100008):
        z = ws.solve(seed, tol=1e-8, warm=False)
        w = ws.solve(seed, tol=1e-8, warm=True)
        assert z["status"] == 0 and w["status"] == 0
        diff = torch.linalg.norm(w["costate"] - z["costate"]) / torch.linalg.norm(z["costate"])
        assert float(diff) <= 1e-6
        zero_its.append(z["iterations"])
        warm_its.append(w["iterations"])
    assert np.mean(warm_its) < np.mean(zero_its)
    ws.close()
