"""FP64 CPU reference of the warm-start network (test infrastructure only).

The learned initial guess of the pressure-increment solve is a plain stack of
3x3 convolutions on the regular background lattice (zero padding, stride 1),
ReLU between layers, no activation after the last one.  This module is the
definition written out in NumPy: forward pass, mean-squared-error loss over the
active lattice points and its gradients by the chain rule, and one Adam update
(Kingma and Ba, 2015).  Only tests, the smoke check and the CPU legs of the
benchmark may import it; the GPU path never does.

Tensor layout: activations [H, W, C] (channels last); weights [3, 3, Cin, Cout]
indexed [dy+1, dx+1, ci, co]; biases [Cout].

Two losses: the mean squared error of the prediction, and a residual proxy, the
squared 5-point lattice Laplacian of the error (what the Poisson residual of the
resulting initial guess measures) plus a small multiple of the squared error.

Pins (tests/test_cnn_oracle.py): the convolution equals an independent direct
sum over taps; the lattice Laplacian equals a loop over points and vanishes on
linear fields away from the image edge; the gradients of both losses equal
central finite differences; one Adam step equals the update written from its
definition.
"""
from __future__ import annotations

import numpy as np


def conv3x3(x, w, b):
    """y[i, j, co] = b[co] + sum_{dy,dx,ci} x[i+dy, j+dx, ci] w[dy+1, dx+1, ci, co] (zero padding)."""
    H, W, _ = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (0, 0)))
    y = np.broadcast_to(b, (H, W, w.shape[3])).astype(np.float64).copy()
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            y += xp[1 + dy:1 + dy + H, 1 + dx:1 + dx + W, :] @ w[dy + 1, dx + 1]
    return y


def conv3x3_backward(x, w, gy):
    """Gradients of conv3x3 w.r.t. its input, weights and bias for upstream gradient gy."""
    H, W, _ = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (0, 0)))
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            xs = xp[1 + dy:1 + dy + H, 1 + dx:1 + dx + W, :]
            gw[dy + 1, dx + 1] = np.einsum("ijc,ijo->co", xs, gy)
            gxp[1 + dy:1 + dy + H, 1 + dx:1 + dx + W, :] += gy @ w[dy + 1, dx + 1].T
    return gxp[1:-1, 1:-1, :], gw, gy.sum(axis=(0, 1))


def forward(params, x):
    """Run the stack; returns the output [H, W, Cout_last] and the per-layer inputs."""
    acts = [x]
    h = x
    n = len(params)
    for k, (w, b) in enumerate(params):
        h = conv3x3(h, w, b)
        if k < n - 1:
            h = np.maximum(h, 0.0)
            acts.append(h)
    return h, acts


def loss(params, x, target, mask):
    """Mean of (output[..., 0] - target)^2 over the lattice points where mask != 0."""
    y, _ = forward(params, x)
    m = mask != 0
    d = (y[..., 0] - target)[m]
    return float(np.mean(d * d))


def loss_and_grads(params, x, target, mask):
    y, acts = forward(params, x)
    m = (mask != 0).astype(np.float64)
    cnt = max(m.sum(), 1.0)
    d = (y[..., 0] - target) * m
    L = float((d * d).sum() / cnt)
    gy = np.zeros_like(y)
    gy[..., 0] = 2.0 * d / cnt
    grads = [None] * len(params)
    for k in range(len(params) - 1, -1, -1):
        w, b = params[k]
        gx, gw, gb = conv3x3_backward(acts[k], w, gy)
        grads[k] = (gw, gb)
        if k > 0:
            gy = gx * (acts[k] > 0)
    return L, grads


def lap5(e):
    """5-point lattice Laplacian in lattice units with zero values outside the image:
    (Delta e)[i, j] = e[i+1, j] + e[i-1, j] + e[i, j+1] + e[i, j-1] - 4 e[i, j]."""
    ep = np.pad(e, 1)
    return ep[2:, 1:-1] + ep[:-2, 1:-1] + ep[1:-1, 2:] + ep[1:-1, :-2] - 4.0 * e


def residual_loss(params, x, target, mask, lam):
    """Residual proxy of an initial guess.  With e = mask (output[..., 0] - target), the
    error the guess leaves at the active points, the solve starts from the residual
    L e (L the Poisson operator, ~ Delta / h^2 on the lattice), so the loss is the
    squared lattice Laplacian of that error plus a small error term:
        (sum over active points of (Delta e)^2 + lam e^2) / (number of active points)."""
    y, _ = forward(params, x)
    m = (mask != 0).astype(np.float64)
    cnt = max(m.sum(), 1.0)
    e = m * (y[..., 0] - target)
    q = m * lap5(e)
    return float(((q * q).sum() + lam * (e * e).sum()) / cnt)


def residual_loss_and_grads(params, x, target, mask, lam):
    """residual_loss and its parameter gradients by the chain rule: with q = m Delta e,
    dL/dy = (2 / cnt) m (Delta q + lam e) (Delta is symmetric on zero-padded images)."""
    y, acts = forward(params, x)
    m = (mask != 0).astype(np.float64)
    cnt = max(m.sum(), 1.0)
    e = m * (y[..., 0] - target)
    q = m * lap5(e)
    L = float(((q * q).sum() + lam * (e * e).sum()) / cnt)
    gy = np.zeros_like(y)
    gy[..., 0] = 2.0 * m * (lap5(q) + lam * e) / cnt
    grads = [None] * len(params)
    for k in range(len(params) - 1, -1, -1):
        w, b = params[k]
        gx, gw, gb = conv3x3_backward(acts[k], w, gy)
        grads[k] = (gw, gb)
        if k > 0:
            gy = gx * (acts[k] > 0)
    return L, grads


def adam_step(p, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update of array p with gradient g and moments m, v at step t (1-based)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(channels=(16, 32, 32, 32, 32, 32, 16), seed=0):
    """He-style random weights for the layer widths given (input, hidden..., output)."""
    rng = np.random.default_rng(seed)
    ps = []
    for ci, co in zip(channels[:-1], channels[1:]):
        w = rng.standard_normal((3, 3, ci, co)) * np.sqrt(2.0 / (9 * ci))
        ps.append((w, np.zeros(co)))
    return ps
