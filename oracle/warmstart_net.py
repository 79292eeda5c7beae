"""CPU oracle for the learned warm start of PCG (the initial iterate
delta^(0) that Algorithm 1 accepts; a zero start is the paper's default).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import this module; the library never does,
and nothing here is shared with the CUDA sources.

The network is a plain stack of 3x3 convolutions over the K x N grid of
subsystems (zero padding, stride 1), ReLU between layers and none after the
last.  Its input at node (i, j) is the initial state x0_{i,j} (n channels)
and the coupling scale c of the instance (one channel, constant over the
grid); its output at (i, j) is the stacked costate guess for that node over
the horizon, (T+1) n channels, scaled by a fixed sigma:

    delta0[t][i N + j][k] = sigma * yhat[t n + k][i][j].

Everything is written from the definitions, in float64:

  * convolution (cross-correlation, the deep-learning convention)
        y[b, o, i, j] = bias[o] + sum_{c, di, dj} w[o, c, di, dj] x[b, c, i+di-1, j+dj-1]
    with x = 0 outside the grid;
  * its gradients by the chain rule;
  * the loss: mean squared error against the scaled target delta*/sigma;
  * Adam (Kingma and Ba, "Adam: a method for stochastic optimization",
    ICLR 2015, Algorithm 1) with bias correction;
  * round-to-nearest-even to bfloat16 (8 significant bits), the storage
    format of the weights in the forward pass.
"""
from __future__ import annotations

import numpy as np


def bf16_round(a):
    """Nearest bfloat16 value (ties to even) of each float32 entry of `a`,
    returned as float64.  bfloat16 keeps the sign, the 8 exponent bits and
    the top 7 stored mantissa bits of an IEEE float32."""
    f = np.asarray(a, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    low = bits & 0xFFFF
    keep = bits >> 16
    lsb = keep & 1
    round_up = (low > 0x8000) | ((low == 0x8000) & (lsb == 1))
    keep = keep + round_up.astype(np.uint64)
    out = (keep << 16).astype(np.uint32).view(np.float32)
    return out.astype(np.float64)


def conv3x3(x, w, bias):
    """Same-size 3x3 cross-correlation with zero padding.
    x [B][Cin][H][W], w [Cout][Cin][3][3], bias [Cout] -> [B][Cout][H][W]."""
    B, Cin, H, W = x.shape
    xp = np.zeros((B, Cin, H + 2, W + 2))
    xp[:, :, 1:H + 1, 1:W + 1] = x
    y = np.broadcast_to(np.asarray(bias, dtype=np.float64)[None, :, None, None],
                        (B, w.shape[0], H, W)).copy()
    for di in range(3):
        for dj in range(3):
            y += np.einsum("oc,bchw->bohw", w[:, :, di, dj], xp[:, :, di:di + H, dj:dj + W])
    return y


def conv3x3_backward(x, w, gy):
    """Gradients of sum(gy * conv3x3(x, w, b)) with respect to x, w and b."""
    B, Cin, H, W = x.shape
    xp = np.zeros((B, Cin, H + 2, W + 2))
    xp[:, :, 1:H + 1, 1:W + 1] = x
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w, dtype=np.float64)
    for di in range(3):
        for dj in range(3):
            win = xp[:, :, di:di + H, dj:dj + W]
            gw[:, :, di, dj] = np.einsum("bohw,bchw->oc", gy, win)
            gxp[:, :, di:di + H, dj:dj + W] += np.einsum("oc,bohw->bchw", w[:, :, di, dj], gy)
    gb = gy.sum(axis=(0, 2, 3))
    return gxp[:, :, 1:H + 1, 1:W + 1], gw, gb


def layer_sizes(n, T, channels, layers):
    """Channel counts of the stack: n + 1 inputs, `channels` in each hidden
    layer, (T + 1) n outputs; `layers` convolutions."""
    return [n + 1] + [channels] * (layers - 1) + [(T + 1) * n]


def forward(params, x):
    """params: list of (w, b) per layer; x [B][C0][H][W].  Returns the output
    and the input of every layer (for the backward pass)."""
    inputs = []
    a = x
    for l, (w, b) in enumerate(params):
        inputs.append(a)
        z = conv3x3(a, w, b)
        a = np.maximum(z, 0.0) if l + 1 < len(params) else z
    return a, inputs


def loss(yhat, target_scaled):
    """Mean squared error over every output entry."""
    d = yhat - target_scaled
    return float(np.mean(d * d))


def loss_and_grads(params, x, target_scaled):
    """Loss and its gradient with respect to every (w, b)."""
    yhat, inputs = forward(params, x)
    g = 2.0 * (yhat - target_scaled) / yhat.size
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        w, _ = params[l]
        gx, gw, gb = conv3x3_backward(inputs[l], w, g)
        grads[l] = (gw, gb)
        if l > 0:
            # the layer input is relu(z) of the layer before: pass where z > 0
            g = gx * (inputs[l] > 0.0)
    return loss(yhat, target_scaled), grads


def adam_step(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1).  Returns new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


def features(x0, c, K, N, n):
    """Network input of one instance: x0 [K*N][n] and the coupling scale c
    -> [n + 1][K][N]."""
    x = np.empty((n + 1, K, N))
    x[:n] = np.asarray(x0, dtype=np.float64).reshape(K, N, n).transpose(2, 0, 1)
    x[n] = c
    return x


def to_delta(yhat, K, N, T, n, sigma):
    """Network output [(T+1) n][K][N] -> delta0 [T+1][K*N][n]."""
    return sigma * np.asarray(yhat).reshape(T + 1, n, K, N).transpose(0, 2, 3, 1).reshape(T + 1, K * N, n)


def from_delta(delta, K, N, T, n, sigma):
    """Inverse of to_delta: the scaled training target."""
    return np.asarray(delta).reshape(T + 1, K, N, n).transpose(0, 3, 1, 2).reshape((T + 1) * n, K, N) / sigma


def predict(params, x0, c, K, N, T, n, sigma):
    """delta0 of one instance, with the weights as given (callers pass the
    bfloat16-rounded weights that the forward pass uses)."""
    yhat, _ = forward(params, features(x0, c, K, N, n)[None])
    return to_delta(yhat[0], K, N, T, n, sigma)
