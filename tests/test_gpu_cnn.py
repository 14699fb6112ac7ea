"""Warm-start network on the GPU vs the FP64 CPU reference (oracle/cnn_oracle.py).

Tolerances: the GPU keeps weights, activations and gradients in BF16 (8-bit
mantissa, relative rounding 2^-9 ~ 2e-3 per value) and accumulates in FP32;
through six layers the relative L2 error of the output stays below ~2e-2.  The
gradients of the lower layers drift further from the FP64 values (ReLU masks
that flip where a pre-activation is within rounding of zero, compounded layer by
layer: ~1e-1 at the first layer for random weights), so the gradient test
compares with the FP64 reference evaluated on the same BF16-rounded weights,
activations and back-propagated gradients (the GPU's storage points), where
only the FP32 summation order differs: bar 1e-2.  Against the pure FP64
gradients only the last two layers are held, at 5e-2.
"""
import numpy as np
import pytest

import workloads as w
from oracle import cnn_oracle as co

pytestmark = pytest.mark.gpu

CH = (16, 32, 32, 32, 32, 32, 1)


def to_layers(flat):
    out, o = [], 0
    for ci, cout in zip(CH[:-1], CH[1:]):
        n = 9 * ci * cout
        wgt = flat[o:o + n].reshape(3, 3, ci, cout).astype(np.float64)
        o += n
        b = flat[o:o + cout].astype(np.float64)
        o += cout
        out.append((wgt, b))
    assert o == flat.size
    return out


def bf16(a):
    a = np.asarray(a, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32)


@pytest.fixture(scope="module")
def ctx(vip):
    c = vip.solver_for(w.cavity(24, Re=100.0), precision=vip.VIP_PREC_FP64)
    c.vip_ws_set_loss(0)  # the tests below compare with the oracle's mean squared error
    yield c
    c.close()


def random_params(ctx, seed):
    import ctypes as C
    n = C.c_int64()
    ctx._check(ctx.L.vip_ws_params(ctx.h, 0, None, C.byref(n)))
    rng = np.random.default_rng(seed)
    flat = np.zeros(n.value, np.float32)
    o = 0
    for ci, cout in zip(CH[:-1], CH[1:]):
        k = 9 * ci * cout
        flat[o:o + k] = rng.standard_normal(k) * np.sqrt(2.0 / (9 * ci))
        o += k
        flat[o:o + cout] = 0.1 * rng.standard_normal(cout)
        o += cout
    ctx._check(ctx.L.vip_ws_params(ctx.h, 1, flat.ctypes.data_as(C.POINTER(C.c_float)), None))
    return flat


def eval_gpu(ctx, x, target=None, mask=None, nparams=None):
    import ctypes as C
    H, W, _ = x.shape
    x = np.ascontiguousarray(x, np.float32)
    y = np.zeros((H, W), np.float32)
    grads = loss = None
    args = [None, None, None, None]
    if target is not None:
        grads = np.zeros(nparams, np.float32)
        loss = C.c_double()
        t = np.ascontiguousarray(target, np.float32)
        m = np.ascontiguousarray(mask, np.float32)
        args = [grads.ctypes.data, t.ctypes.data, m.ctypes.data, C.byref(loss)]
    ctx._check(ctx.L.vip_ws_eval(ctx.h, H, W, x.ctypes.data, y.ctypes.data, *args))
    return y, grads, (loss.value if loss is not None else None)


@pytest.mark.parametrize("shape", [(3, 5), (6, 150), (2, 300)])
def test_forward_matches_reference(ctx, shape):
    flat = random_params(ctx, 1)
    rng = np.random.default_rng(2)
    H, W = shape
    x = np.zeros((H, W, 16), np.float32)
    x[..., :6] = rng.standard_normal((H, W, 6))
    x = bf16(x)
    y, _, _ = eval_gpu(ctx, x)
    ref, _ = co.forward(to_layers(flat), x.astype(np.float64))
    ref = ref[..., 0]
    err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert err < 2e-2, err


def bf16_reference_grads(layers, x, t, m, lam=None):
    """FP64 forward/backward of the oracle with BF16 rounding where the GPU stores
    BF16: packed weights, ReLU outputs, the loss gradient and each data gradient.
    lam None: mean squared error; else the residual proxy with that weight."""
    wq = [(bf16(wt).astype(np.float64), b) for wt, b in layers]
    acts, h = [x], x
    for k, (wt, b) in enumerate(wq):
        h = co.conv3x3(h, wt, b)
        if k < len(wq) - 1:
            h = bf16(np.maximum(h, 0.0)).astype(np.float64)
            acts.append(h)
    y = h[..., 0].astype(np.float32).astype(np.float64)
    d = (y - t) * m
    gy = np.zeros(h.shape)
    if lam is None:
        gy[..., 0] = bf16(2.0 * d / max(m.sum(), 1.0))
    else:
        q = (m * co.lap5(d)).astype(np.float32).astype(np.float64)
        gy[..., 0] = bf16(2.0 * m * (co.lap5(q) + lam * d) / max(m.sum(), 1.0))
    out = [None] * len(wq)
    for k in range(len(wq) - 1, -1, -1):
        gx, gw, gb = co.conv3x3_backward(acts[k], wq[k][0], gy)
        out[k] = (gw, gb)
        if k > 0:
            gy = bf16(gx * (acts[k] > 0)).astype(np.float64)
    return out


def test_gradients_match_reference(ctx):
    flat = random_params(ctx, 3)
    rng = np.random.default_rng(4)
    H, W = 5, 140
    x = np.zeros((H, W, 16), np.float32)
    x[..., :6] = rng.standard_normal((H, W, 6))
    x = bf16(x)
    t = rng.standard_normal((H, W)).astype(np.float32)
    m = (rng.random((H, W)) > 0.2).astype(np.float32)
    _, g, loss = eval_gpu(ctx, x, t, m, flat.size)
    layers = to_layers(flat)
    x64, t64, m64 = x.astype(np.float64), t.astype(np.float64), m.astype(np.float64)
    L, ref = co.loss_and_grads(layers, x64, t64, m64)
    emu = bf16_reference_grads(layers, x64, t64, m64)
    assert abs(loss - L) <= 2e-2 * abs(L)
    o = 0
    for k, (ci, cout) in enumerate(zip(CH[:-1], CH[1:])):
        n = 9 * ci * cout
        got_w = g[o:o + n].reshape(ref[k][0].shape)
        o += n
        got_b = g[o:o + cout]
        o += cout

        def rel(a, b):
            return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        ew, eb = rel(got_w, emu[k][0]), rel(got_b, emu[k][1])
        assert ew < 1e-2 and eb < 1e-2, (k, ci, cout, ew, eb)
        if k >= len(CH) - 3:
            ew, eb = rel(got_w, ref[k][0]), rel(got_b, ref[k][1])
            assert ew < 5e-2 and eb < 5e-2, (k, ci, cout, ew, eb)


def test_residual_loss_gradients_match_reference(ctx):
    """The residual-proxy loss (squared lattice Laplacian of the error plus lam times
    the squared error) and its parameter gradients against the oracle: the loss
    within 2e-2 of FP64, the gradients within 1e-2 of the oracle evaluated at the
    GPU's BF16 storage points, as for the mean squared error."""
    lam = 0.05
    flat = random_params(ctx, 8)
    rng = np.random.default_rng(9)
    H, W = 6, 130
    x = np.zeros((H, W, 16), np.float32)
    x[..., :6] = rng.standard_normal((H, W, 6))
    x = bf16(x)
    t = rng.standard_normal((H, W)).astype(np.float32)
    m = (rng.random((H, W)) > 0.2).astype(np.float32)
    ctx.vip_ws_set_loss(1, lam)
    try:
        _, g, loss = eval_gpu(ctx, x, t, m, flat.size)
    finally:
        ctx.vip_ws_set_loss(0)
    layers = to_layers(flat)
    x64, t64, m64 = x.astype(np.float64), t.astype(np.float64), m.astype(np.float64)
    L, _ = co.residual_loss_and_grads(layers, x64, t64, m64, lam)
    emu = bf16_reference_grads(layers, x64, t64, m64, lam)
    assert abs(loss - L) <= 2e-2 * abs(L)
    o = 0
    for k, (ci, cout) in enumerate(zip(CH[:-1], CH[1:])):
        n = 9 * ci * cout
        got_w = g[o:o + n].reshape(emu[k][0].shape)
        o += n
        got_b = g[o:o + cout]
        o += cout
        rel = lambda a, b: np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)  # noqa: E731
        assert rel(got_w, emu[k][0]) < 1e-2 and rel(got_b, emu[k][1]) < 1e-2, k


def test_adam_matches_oracle(ctx):
    """Three Adam updates on the GPU (vip_ws_adam after vip_ws_eval on three different
    images) against the oracle's adam_step (oracle/cnn_oracle.py) fed the same
    gradients, from the same parameters and zero moments, element by element.  The
    GPU keeps parameters, moments and the update in FP32 (bias corrections by powf):
    after each update |p_gpu - p_oracle| <= 2^-22 |p| (two FP32 roundings of p)
    + 1e-5 lr (FP32 arithmetic in the update)."""
    lr = 1e-3
    flat = random_params(ctx, 5)  # loading the parameters zeroes the moments and the step count
    rng = np.random.default_rng(6)
    H, W = 4, 96
    p = flat.astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for t in (1, 2, 3):
        x = np.zeros((H, W, 16), np.float32)
        x[..., :6] = rng.standard_normal((H, W, 6))
        x = bf16(x)
        tgt = rng.standard_normal((H, W)).astype(np.float32)
        msk = (rng.random((H, W)) > 0.3).astype(np.float32)
        _, g, _ = eval_gpu(ctx, x, tgt, msk, flat.size)
        ctx.vip_ws_adam(lr)
        got = ctx.vip_ws_params().astype(np.float64)
        p, m, v = co.adam_step(p, g.astype(np.float64), m, v, t, lr=lr)
        bar = 2.0 ** -22 * np.abs(p) + 1e-5 * lr
        assert np.all(np.abs(got - p) <= bar), (t, np.max(np.abs(got - p) - bar))
        p = got  # continue from the GPU's FP32 parameters, as the GPU does


def test_untrained_network_reproduces_previous_increment_guess(vip):
    """With the untrained (zero last layer) network the warm start equals the plain
    previous-increment guess, so the state matches the run without it."""
    ns = w.cavity(32, Re=400.0)
    a = vip.solver_for(ns, precision=vip.VIP_PREC_FP64, rtol=1e-12)
    b = vip.solver_for(ns, precision=vip.VIP_PREC_FP64, rtol=1e-12)
    b._check(b.L.vip_ws_enable(b.h, 1))
    a.vip_step(5)
    b.vip_step(5)
    ua = a.vip_get_state()
    ub = b.vip_get_state()
    for x, y in zip(ua, ub):
        assert np.allclose(x, y, rtol=0, atol=1e-10 * max(1.0, np.max(np.abs(y))))
    a.close()
    b.close()


def test_collect_train_and_use(vip):
    """Collect solver-generated samples, train, and step with the learned guess: the
    training loss falls and the solution is unchanged to the solver tolerance."""
    import ctypes as C
    ns = w.cavity(48, Re=400.0)
    ref = vip.solver_for(ns, precision=vip.VIP_PREC_FP64, rtol=1e-10)
    ctx = vip.solver_for(ns, precision=vip.VIP_PREC_FP64, rtol=1e-10)
    ctx.vip_step(10)
    ref.vip_step(10)
    ctx._check(ctx.L.vip_ws_collect(ctx.h, 1, 20))
    ctx.vip_step(20)
    ref.vip_step(20)
    ctx._check(ctx.L.vip_ws_collect(ctx.h, 0, 0))
    cfg = vip.TrainCfg(epochs=8, lr=1e-3, seed=7)
    ctx._check(ctx.L.vip_ws_train(ctx.h, C.byref(cfg)))
    assert cfg.final_loss < cfg.first_loss
    ctx._check(ctx.L.vip_ws_enable(ctx.h, 1))
    ctx.vip_step(5)
    ref.vip_step(5)
    u1, v1, p1, _ = ctx.vip_get_state()
    u0, v0, p0, _ = ref.vip_get_state()
    assert np.linalg.norm(u1 - u0) <= 1e-6 * np.linalg.norm(u0)
    assert np.linalg.norm(p1 - p0) <= 1e-6 * np.linalg.norm(p0)
    ctx.close()
    ref.close()
