"""The multigrid's cell-grid parity (vip_set_mg_shift) on the GPU.

Level 1 of the Poisson preconditioner aggregates 2h x 2h cells of the background
lattice; a shift of one lattice spacing pairs different rows and columns.  On a
channel, shifting by one row pairs a slip-wall row with the first interior row, a
far weaker hierarchy: the solve needs more iterations (about ten times as many on
this case, from the same hierarchy assembled on the host from the oracle's
operators).  The parity changes only the iteration count: every solve still stops
at its residual, recomputed here on the host from the exported operator.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as w

pytestmark = pytest.mark.gpu


def test_cell_grid_shift_changes_convergence_not_the_solve(vip):
    ns = w.channel_body(1 / 16, ("circle", 0.5), Re=100.0, xlim=(-4, 8), ylim=(-3, 3))
    rng = np.random.default_rng(7)
    b = np.where(ns.kind == 0, rng.standard_normal(ns.n), 0.0)
    its = {}
    for shift in ((0, 0), (0, 1), (1, 0)):
        ctx = vip.solver_for(ns, precision=vip.VIP_PREC_FP64, rtol=1e-10, mg_shifts=[shift])
        ptr, col, val = ctx.vip_get_stencil("POISSON")
        P = sp.csr_matrix((val, col, ptr), shape=(ns.n, ns.n))
        x, it, rr = ctx.vip_solve("POISSON", b, np.zeros(ns.n), precision=vip.VIP_PREC_FP64,
                                  rtol=1e-10, max_iters=5000)
        ctx.close()
        assert rr <= 1e-10, (shift, rr)
        assert np.linalg.norm(b - P @ x) <= 1.01e-10 * np.linalg.norm(b), shift
        its[shift] = it
    assert its[(0, 1)] > its[(0, 0)], its


def test_cell_grid_shift_arguments(vip):
    ns = w.cavity(16, Re=100.0)
    ctx = vip.Context()
    ctx.add_nodeset(ns)
    for bad in ((5, 0, 0), (0, 2, 0), (0, 0, -1)):
        with pytest.raises(vip.VipError):
            ctx.vip_set_mg_shift(*bad)
    ctx.vip_set_mg_shift(-1, 1, 1)
    ctx.close()
    box = vip.Context()
    box.add_nodeset(w.periodic_box(16))
    with pytest.raises(vip.VipError):      # a periodic axis keeps 0
        box.vip_set_mg_shift(0, 1, 0)
    box.close()
