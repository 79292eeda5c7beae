"""Pins of the warm-start network oracle against facts outside itself:
SciPy's 2D correlation, impulse responses, central finite differences,
closed forms of Adam's first steps, the definition of bfloat16 rounding and
the stated index maps."""
import numpy as np
from scipy import signal

from oracle import warmstart_net as W


def rng(seed=0):
    return np.random.default_rng(seed)


def test_conv_matches_scipy_correlate2d():
    r = rng(1)
    x = r.standard_normal((2, 3, 7, 5))
    w = r.standard_normal((4, 3, 3, 3))
    b = r.standard_normal(4)
    y = W.conv3x3(x, w, b)
    for bb in range(2):
        for o in range(4):
            ref = b[o] + sum(signal.correlate2d(x[bb, c], w[o, c], mode="same", boundary="fill", fillvalue=0.0)
                             for c in range(3))
            assert np.allclose(y[bb, o], ref, rtol=1e-13, atol=1e-13)


def test_conv_impulse_response_is_the_flipped_kernel():
    w = np.arange(9.0).reshape(1, 1, 3, 3) + 1.0
    x = np.zeros((1, 1, 5, 5))
    x[0, 0, 2, 2] = 1.0
    y = W.conv3x3(x, w, np.zeros(1))[0, 0]
    # output (i, j) sees the impulse at (2, 2) through tap (3 - i, 3 - j), so
    # the 3 x 3 window around it holds the kernel flipped in both axes
    assert np.array_equal(y[1:4, 1:4], w[0, 0, ::-1, ::-1])
    assert y.sum() == w.sum()


def test_conv_of_constant_interior_sums_taps_and_edges_drop_taps():
    w = rng(2).standard_normal((1, 1, 3, 3))
    y = W.conv3x3(np.ones((1, 1, 4, 4)), w, np.zeros(1))[0, 0]
    assert np.isclose(y[1, 1], w.sum())
    assert np.isclose(y[0, 0], w[0, 0, 1:, 1:].sum())


def tiny_net(seed=3, n=2, T=1, ch=4, layers=3):
    r = rng(seed)
    sizes = W.layer_sizes(n, T, ch, layers)
    return [(r.standard_normal((sizes[l + 1], sizes[l], 3, 3)) * 0.4, r.standard_normal(sizes[l + 1]) * 0.1)
            for l in range(layers)], sizes


def test_gradients_match_central_differences():
    params, sizes = tiny_net()
    r = rng(4)
    x = r.standard_normal((2, sizes[0], 4, 5))
    tgt = r.standard_normal((2, sizes[-1], 4, 5))
    L, grads = W.loss_and_grads(params, x, tgt)
    h = 1e-6
    for l, (w, b) in enumerate(params):
        for arr, g in ((w, grads[l][0]), (b, grads[l][1])):
            flat = arr.reshape(-1)
            idx = r.choice(flat.size, size=min(6, flat.size), replace=False)
            for e in idx:
                old = flat[e]
                flat[e] = old + h
                lp = W.loss(W.forward(params, x)[0], tgt)
                flat[e] = old - h
                lm = W.loss(W.forward(params, x)[0], tgt)
                flat[e] = old
                fd = (lp - lm) / (2 * h)
                assert abs(g.reshape(-1)[e] - fd) <= 1e-6 * max(1.0, abs(fd)), (l, e)


def test_relu_gate_uses_the_preactivation_sign():
    # with all-negative biases and zero weights in layer 0, nothing passes
    params, sizes = tiny_net()
    w0, _ = params[0]
    params[0] = (np.zeros_like(w0), -np.ones(sizes[1]))
    x = rng(5).standard_normal((1, sizes[0], 3, 3))
    _, grads = W.loss_and_grads(params, x, np.zeros((1, sizes[-1], 3, 3)))
    assert np.all(grads[0][0] == 0.0) and np.all(grads[0][1] == 0.0)


def test_adam_first_step_and_constant_gradient():
    g = np.array([0.3, -2.0, 1e-3])
    p = np.array([1.0, 2.0, 3.0])
    lr, eps = 1e-2, 1e-8
    p1, m, v = W.adam_step(p, g, np.zeros(3), np.zeros(3), 1, lr, eps=eps)
    # bias correction makes m_hat = g and v_hat = g^2 on the first step
    assert np.allclose(p1, p - lr * g / (np.abs(g) + eps), rtol=1e-14)
    q = p1
    for step in range(2, 6):
        q_new, m, v = W.adam_step(q, g, m, v, step, lr, eps=eps)
        assert np.allclose(q - q_new, lr * g / (np.abs(g) + eps), rtol=1e-12)
        q = q_new


def test_bf16_rounding_definition():
    exact = np.array([1.0, -2.5, 0.0, 3.0 * 2.0 ** -20, 65280.0])
    assert np.array_equal(W.bf16_round(exact), exact)
    one = 1.0
    ulp = 2.0 ** -7                       # spacing of bfloat16 just above 1
    assert W.bf16_round(one + ulp / 2) == one            # tie -> even (1.0)
    assert W.bf16_round(one + 1.5 * ulp) == one + 2 * ulp  # tie -> even (1 + 2 ulp)
    assert W.bf16_round(one + 0.51 * ulp) == one + ulp
    x = rng(6).standard_normal(10000).astype(np.float32)
    rel = np.abs(W.bf16_round(x) - x) / np.abs(x)
    assert rel.max() <= 2.0 ** -8 * (1 + 1e-6)


def test_feature_and_output_index_maps():
    K, N, T, n = 3, 4, 2, 2
    r = rng(7)
    x0 = r.standard_normal((K * N, n))
    f = W.features(x0, 0.25, K, N, n)
    assert f[1, 2, 3] == x0[2 * N + 3, 1] and np.all(f[n] == 0.25)
    delta = r.standard_normal((T + 1, K * N, n))
    yhat = W.from_delta(delta, K, N, T, n, 2.0)
    t, i, j, k = 2, 1, 3, 1
    assert yhat[t * n + k, i, j] * 2.0 == delta[t, i * N + j, k]
    assert np.array_equal(W.to_delta(yhat, K, N, T, n, 2.0), delta)


def test_gradient_vanishes_at_an_exact_fit():
    """A one-layer (linear) net whose weights generated the target has zero
    loss, and the gradient there is zero (first-order optimality)."""
    r = rng(8)
    x = r.standard_normal((3, 2, 4, 4))
    w_true = r.standard_normal((3, 2, 3, 3))
    b_true = r.standard_normal(3)
    tgt = W.conv3x3(x, w_true, b_true)
    L, grads = W.loss_and_grads([(w_true, b_true)], x, tgt)
    assert L == 0.0
    assert np.abs(grads[0][0]).max() == 0.0 and np.abs(grads[0][1]).max() == 0.0
