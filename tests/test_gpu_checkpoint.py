"""Checkpoint and resume through the C ABI (vip_checkpoint_size, vip_checkpoint).

A checkpoint holds everything the next fractional step depends on (u, v, p, the
last increment phi, the Adams-Bashforth history N^{n-1} of Eq. 12, the held
Dirichlet values and the step counter).  The kernels reduce in a fixed order, so
the steps after a restore must repeat the steps after the save bit for bit, in
every precision form.  A buffer whose checksum does not match, or that belongs to
a context of other sizes, is refused and leaves the state untouched."""
import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu


def state(ctx):
    return ctx.vip_get_state()


@pytest.mark.parametrize("form", ["FP64", "MIXED"])
def test_restore_repeats_the_steps_bitwise(vip, form):
    prec = vip.VIP_PREC_FP64 if form == "FP64" else vip.VIP_PREC_MIXED
    ctx = vip.solver_for(w.cavity(24, Re=400.0), precision=prec, rtol=1e-8)
    ctx.vip_step(3)  # past the Euler start, so the history N^{n-1} matters
    buf = ctx.vip_checkpoint(True)
    ctx.vip_step(4)
    first = state(ctx)
    it0 = ctx.vip_get_stats().total_poisson_iters
    ctx.vip_checkpoint(False, buf)
    ctx.vip_step(4)
    again = state(ctx)
    it1 = ctx.vip_get_stats().total_poisson_iters
    for a, b in zip(first, again):
        assert np.array_equal(a, b)
    assert it1 - it0 > 0
    ctx.close()


def test_device_buffer_and_refusals(vip):
    torch = pytest.importorskip("torch")
    ns = w.channel_body(1 / 8, ("circle", 0.5), Re=100.0, xlim=(-3, 5), ylim=(-2, 2))
    ctx = vip.solver_for(ns, precision=vip.VIP_PREC_FP64, rtol=1e-10)
    ctx.vip_step(2)
    n = ctx.vip_checkpoint_size()
    dbuf = torch.zeros(n, dtype=torch.uint8, device="cuda")
    ctx.vip_checkpoint(True, dbuf)
    hbuf = dbuf.cpu().numpy().copy()
    ctx.vip_step(3)
    first = state(ctx)
    ctx.vip_checkpoint(False, dbuf)
    ctx.vip_step(3)
    for a, b in zip(first, state(ctx)):
        assert np.array_equal(a, b)
    # a flipped byte in the body: refused, state unchanged
    bad = hbuf.copy()
    bad[n // 2] ^= 0x40
    before = state(ctx)
    with pytest.raises(vip.VipError) as e:
        ctx.vip_checkpoint(False, bad)
    assert e.value.status == vip.VIP_ERR_ARG
    for a, b in zip(before, state(ctx)):
        assert np.array_equal(a, b)
    # a checkpoint of another context's sizes: refused
    other = vip.solver_for(w.cavity(16, Re=100.0), precision=vip.VIP_PREC_FP64)
    obuf = other.vip_checkpoint(True)
    with pytest.raises(vip.VipError):
        ctx.vip_checkpoint(False, np.resize(obuf, n))
    other.close()
    # the host copy of the device checkpoint restores the same state
    ctx.vip_checkpoint(False, hbuf)
    ctx.vip_step(3)
    for a, b in zip(first, state(ctx)):
        assert np.array_equal(a, b)
    ctx.close()
