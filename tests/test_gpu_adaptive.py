"""Stepwise adaptive node distributions (workloads.channel_body(refine=...)) through
the C ABI.

Parity with the oracle on a small adaptive channel (h = 1/8 in a box, 1/4
outside): neighbour lists exact, MLS weights and merged operators to 1e-10, and
ten all-FP64 fractional steps to 1e-10 relative L2 with both sides' solves at
1e-13 (the bars of tests/test_gpu_parity.py).
(The multigrid's cell lattice is at the finest spacing and its Galerkin stencils
reach two cells, so in the coarse regions, where nodes lie four or more cells
apart, couplings are lost and the preconditioner degrades: an FP64 solve on a
spacing 1/64 ... 1/8 channel took 1,744 iterations.  Large adaptive sets need a
per-region aggregation first.)
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as w
from oracle import vip_oracle as vo

pytestmark = pytest.mark.gpu


def gpu_csr(ctx, which, shape):
    ptr, col, val = ctx.vip_get_stencil(which)
    return sp.csr_matrix((val, col, ptr), shape=shape)


def rel_diff(a, b):
    d = abs(sp.csr_matrix(a) - sp.csr_matrix(b)).max()
    return d / max(abs(sp.csr_matrix(b)).max(), 1e-300)


def small():
    return w.channel_body(1 / 8, ("circle", 0.5), Re=20.0, xlim=(-4, 8), ylim=(-3, 3),
                          refine=[(-1.5, 3.0, -1.5, 1.5)])


def test_small_adaptive_channel_matches_oracle(vip):
    ns = small()
    ctx = vip.solver_for(ns, precision=vip.VIP_PREC_FP64, rtol=1e-13)
    ops = vo.Operators(ns)
    fs = vo.FractionalStep(ops, rtol=1e-13)
    ptr, col, _ = ctx.vip_get_stencil("NBR")
    assert np.array_equal(ptr, ops.node_ptr) and np.array_equal(col.astype(np.int64), ops.node_idx)
    for which, d in (("D00", (0, 0)), ("D10", (1, 0)), ("D20", (2, 0)), ("D02", (0, 2))):
        assert rel_diff(gpu_csr(ctx, which, (ns.n, ns.n)), ops.D[d]) <= 1e-10, which
    for which, ref in (("LAPLACE", ops.L), ("VIP_E", ops.I["e"]), ("GX", ops.Gx), ("GY", ops.Gy),
                       ("HELM_U", fs.Hu), ("POISSON", fs.P)):
        assert rel_diff(gpu_csr(ctx, which, ref.shape), ref) <= 1e-10, which
    ctx.vip_step(10)
    assert ctx.vip_get_stats().status == 0
    for _ in range(10):
        fs.step()
    u, v, p, _ = ctx.vip_get_state()
    for a, b, f in ((u, fs.u, "u"), (v, fs.v, "v"), (p, fs.p, "p")):
        e = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
        assert e <= 1e-10, (f, e)
    ctx.close()
