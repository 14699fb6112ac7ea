"""Pins of the FP64 reference of the warm-start network (CPU only)."""
import numpy as np

from oracle import cnn_oracle as co


def direct_conv(x, w, b):
    """Independent definition: explicit loops over output pixels and taps."""
    H, W, ci = x.shape
    out = np.zeros((H, W, w.shape[3]))
    for i in range(H):
        for j in range(W):
            acc = b.astype(np.float64).copy()
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    ii, jj = i + dy, j + dx
                    if 0 <= ii < H and 0 <= jj < W:
                        acc += x[ii, jj] @ w[dy + 1, dx + 1]
            out[i, j] = acc
    return out


def test_conv_matches_direct_sum():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((5, 7, 3))
    w = rng.standard_normal((3, 3, 3, 4))
    b = rng.standard_normal(4)
    assert np.allclose(co.conv3x3(x, w, b), direct_conv(x, w, b), rtol=0, atol=1e-12)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    params = co.init_params(channels=(4, 5, 5, 2), seed=2)
    x = rng.standard_normal((6, 5, 4))
    t = rng.standard_normal((6, 5))
    mask = (rng.random((6, 5)) > 0.3).astype(float)
    L, grads = co.loss_and_grads(params, x, t, mask)
    assert abs(L - co.loss(params, x, t, mask)) < 1e-14
    eps = 1e-6
    for k, (w, b) in enumerate(params):
        for arr, g in ((w, grads[k][0]), (b, grads[k][1])):
            flat = arr.reshape(-1)
            gflat = g.reshape(-1)
            for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + eps
                lp = co.loss(params, x, t, mask)
                flat[idx] = old - eps
                lm = co.loss(params, x, t, mask)
                flat[idx] = old
                fd = (lp - lm) / (2 * eps)
                assert abs(fd - gflat[idx]) <= 1e-6 * max(1.0, abs(fd)), (k, idx, fd, gflat[idx])


def test_adam_step_definition():
    p = np.array([1.0, -2.0])
    g = np.array([0.5, 0.25])
    p1, m, v = co.adam_step(p, g, np.zeros(2), np.zeros(2), 1, lr=0.1)
    # first step: m_hat = g, v_hat = g^2, update = lr * g / (|g| + eps)
    assert np.allclose(p1, p - 0.1 * g / (np.abs(g) + 1e-8))


def test_lattice_laplacian():
    rng = np.random.default_rng(3)
    e = rng.standard_normal((5, 6))
    ref = np.zeros_like(e)
    for i in range(5):
        for j in range(6):
            acc = -4.0 * e[i, j]
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                if 0 <= i + di < 5 and 0 <= j + dj < 6:
                    acc += e[i + di, j + dj]
            ref[i, j] = acc
    assert np.allclose(co.lap5(e), ref, rtol=0, atol=1e-14)
    ii, jj = np.meshgrid(np.arange(7), np.arange(8), indexing="ij")
    lin = 0.3 * ii - 1.7 * jj + 2.0
    assert np.allclose(co.lap5(lin)[1:-1, 1:-1], 0.0, atol=1e-13)


def test_residual_loss_gradients_match_finite_differences():
    rng = np.random.default_rng(4)
    params = co.init_params(channels=(4, 5, 5, 2), seed=5)
    x = rng.standard_normal((6, 7, 4))
    t = rng.standard_normal((6, 7))
    mask = (rng.random((6, 7)) > 0.3).astype(float)
    lam = 0.05
    L, grads = co.residual_loss_and_grads(params, x, t, mask, lam)
    assert abs(L - co.residual_loss(params, x, t, mask, lam)) < 1e-13
    eps = 1e-6
    for k, (w, b) in enumerate(params):
        for arr, g in ((w, grads[k][0]), (b, grads[k][1])):
            flat = arr.reshape(-1)
            gflat = g.reshape(-1)
            for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + eps
                lp = co.residual_loss(params, x, t, mask, lam)
                flat[idx] = old - eps
                lm = co.residual_loss(params, x, t, mask, lam)
                flat[idx] = old
                fd = (lp - lm) / (2 * eps)
                assert abs(fd - gflat[idx]) <= 1e-6 * max(1.0, abs(fd)), (k, idx, fd, gflat[idx])
