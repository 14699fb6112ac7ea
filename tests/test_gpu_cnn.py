"""Warm-start network on the GPU vs the FP64 CPU reference (oracle/cnn_oracle.py).

Tolerances: the GPU keeps activations and gradients in BF16 (8-bit mantissa,
relative rounding 2^-9 ~ 2e-3 per value) and accumulates in FP32; through six
layers the relative L2 error of the output stays below ~2e-2 and that of the
parameter gradients below ~5e-2.  The bars are set there.
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
    L, ref = co.loss_and_grads(layers, x.astype(np.float64), t.astype(np.float64), m)
    assert abs(loss - L) <= 2e-2 * abs(L)
    o = 0
    for (gw, gb), (ci, cout) in zip(ref, zip(CH[:-1], CH[1:])):
        n = 9 * ci * cout
        got_w = g[o:o + n].reshape(gw.shape)
        o += n
        got_b = g[o:o + cout]
        o += cout
        ew = np.linalg.norm(got_w - gw) / max(np.linalg.norm(gw), 1e-30)
        eb = np.linalg.norm(got_b - gb) / max(np.linalg.norm(gb), 1e-30)
        assert ew < 5e-2 and eb < 5e-2, (ci, cout, ew, eb)


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
