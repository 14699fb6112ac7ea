"""Uniform-slice storage of the Krylov operators (vip_operator_layout), through the
C ABI.  A slice whose 32 rows hold the same stencil bit for bit is applied from
one stored copy, shared by every slice with the same stencil; on a dyadic lattice (h = 2^-k, coordinates exact in binary) the
MLS weights of interior nodes come out bit-identical, so most slices qualify; on
a lattice whose coordinates are not exact in binary few do.  The Krylov solves
through this storage are checked against direct solves and the oracle in
test_gpu_multigrid.py and test_gpu_parity.py."""
import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu


def layout_ok(ctx, which):
    lay = ctx.vip_operator_layout(which)
    ptr, _, _ = ctx.vip_get_stencil(which)
    nnz = int(ptr[-1])
    assert 0 <= lay["uniform_slices"] <= lay["slices"]
    assert lay["other_entries"] % 32 == 0
    # uniform slices read a table of distinct stencils: non-empty exactly when some
    # slice is uniform, and never more entries than the operator has
    assert (lay["uniform_entries"] > 0) == (lay["uniform_slices"] > 0)
    assert lay["uniform_entries"] <= nnz
    return lay


def test_dyadic_lattice_is_mostly_uniform(vip):
    # rows of 513 nodes: only the slices holding a row's two wall nodes, and those
    # next to the body, differ from row to row
    ns = w.channel_body(1 / 16, ("circle", 0.5), Re=100.0)
    ctx = vip.solver_for(ns, precision=vip.VIP_PREC_FP64)
    lay = layout_ok(ctx, "POISSON")
    assert lay["uniform_slices"] >= 0.8 * lay["slices"], lay
    # one stored stencil instead of 32 rows: the streamed entries shrink accordingly
    assert lay["other_entries"] + lay["uniform_entries"] < 0.3 * int(ctx.vip_get_stencil("POISSON")[0][-1])
    # slices with the same stencil share one copy: far fewer distinct stencil entries
    # than one 13-point copy per uniform slice
    assert lay["uniform_entries"] < 0.05 * 13 * lay["uniform_slices"], lay
    lh = layout_ok(ctx, "HELM_U")
    assert lh == ctx.vip_operator_layout("HELM_V")  # one table for both components
    assert lh["uniform_slices"] > 0
    with pytest.raises(vip.VipError):
        ctx.vip_operator_layout("GX")  # not a Krylov operator
    ctx.close()


def test_inexact_coordinates_give_few_uniform_slices(vip):
    ns = w.triangle_cavity(30, Re=100.0)  # h = 1/29: coordinates not exact in binary
    ctx = vip.solver_for(ns, precision=vip.VIP_PREC_FP64)
    lay = layout_ok(ctx, "POISSON")
    assert lay["uniform_slices"] <= 0.25 * lay["slices"], lay
    ctx.vip_step(2)
    assert ctx.vip_get_stats().status == 0
    ctx.close()
