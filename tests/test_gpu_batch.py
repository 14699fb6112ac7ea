"""Several geometries in one context (one persistent Krylov launch per system kind
solves all of them, one graph per step) vs the FP64 oracle run on each geometry
alone.

The batch mixes closed geometries (bordered Poisson: an equilateral and a square
cavity), an open channel with a body and geometries of different sizes, so that
the per-system scalars, the block-to-system map of the Krylov launch, the bordered
rows and the per-geometry multigrid lattices are all exercised.  Tolerance as in
the single-geometry parity tests: both sides solve to relative residual 1e-13,
the states agree to relative L2 1e-10.
"""
import numpy as np
import pytest

import workloads as w
from oracle import vip_oracle as vo

pytestmark = pytest.mark.gpu


def batch():
    return [w.triangle_cavity(33, Re=300.0, name="triangle33"),
            w.cavity(20, Re=1000.0),
            w.channel_body(1 / 8, ("circle", 0.5), Re=100.0, xlim=(-3, 5), ylim=(-2, 2)),
            w.triangle_cavity(45, Re=800.0, name="triangle45")]


def split(a, sizes):
    out, o = [], 0
    for n in sizes:
        out.append(a[o:o + n])
        o += n
    return out


def test_batch_matches_oracle_per_geometry(vip):
    nss = batch()
    ctx = vip.solver_for(nss, precision=vip.VIP_PREC_FP64, rtol=1e-13)
    n, g = ctx.sizes()
    assert n == sum(ns.n for ns in nss) and g == len(nss)
    nsteps = 6
    ctx.vip_step(nsteps)
    st = ctx.vip_get_stats()
    assert st.status == 0
    # per-geometry work counts: every system iterated, none more than the lock-step maximum
    gi = ctx.vip_get_geometry_iters()
    assert gi.shape == (len(nss),) and np.all(gi > 0) and gi.max() <= st.total_poisson_iters
    u, v, p, _ = ctx.vip_get_state()
    sizes = [ns.n for ns in nss]
    for ns, ug, vg, pg in zip(nss, split(u, sizes), split(v, sizes), split(p, sizes)):
        fs = vo.FractionalStep(vo.Operators(ns), rtol=1e-13)
        for _ in range(nsteps):
            fs.step()
        for a, b, f in ((ug, fs.u, "u"), (vg, fs.v, "v"), (pg, fs.p, "p")):
            e = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
            assert e <= 1e-10, (ns.name, f, e)
    ctx.close()


def test_batch_equals_geometries_alone(vip):
    """Batched and single-geometry contexts take the same steps: the states agree to
    the solver tolerance (1e-8 production setting; each system stops on its own
    residual, so iteration counts may differ by a few)."""
    nss = batch()
    ctx = vip.solver_for(nss, precision=vip.VIP_PREC_FP64, rtol=1e-10)
    ctx.vip_step(4)
    u, v, p, _ = ctx.vip_get_state()
    sizes = [ns.n for ns in nss]
    for ns, ug, pg in zip(nss, split(u, sizes), split(p, sizes)):
        one = vip.solver_for(ns, precision=vip.VIP_PREC_FP64, rtol=1e-10)
        one.vip_step(4)
        u1, _, p1, _ = one.vip_get_state()
        one.close()
        assert np.linalg.norm(ug - u1) <= 1e-8 * np.linalg.norm(u1), ns.name
        assert np.linalg.norm(pg - p1) <= 1e-6 * np.linalg.norm(p1), ns.name
    ctx.close()
