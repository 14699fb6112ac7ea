"""The bench workload at its full size (bumpy cylinder in the channel
[-8,24]x[-8,8], h = 1/64, 2,087,551 nodes), in the bench's launch configuration
(one persistent launch of one 1024-thread CTA per SM per Krylov solve, multigrid
preconditioner, uniform-slice operator storage), checked where the oracle can
follow at this size:

  * the MLS Laplacian rows (Eq. vip:1, Sec. 3) of a seeded sample of nodes —
    interior lattice nodes, lattice nodes next to the body, channel-wall nodes and
    body-surface nodes — computed by the oracle for those nodes alone, from their
    own neighbour lists, against the GPU's table rows: columns among the node's
    neighbours, values within 1e-10 of the row's largest entry (the small-case
    parity bar);
  * a Poisson solve (Eq. 13) to relative residual 1e-8 through the production
    Krylov path, its residual recomputed on the host from the exported operator,
    a property that holds at any size;
  * two fractional steps of the bench workload: device status 0, every Poisson
    solve stopped on the FP64 true residual <= 1e-8, finite fields.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as w
from oracle import vip_oracle as vo

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full(vip):
    ns = w.workload("bumpy_h64")
    ctx = vip.solver_for(ns, precision=vip.VIP_PREC_FP64, rtol=1e-8)
    yield ns, ctx
    ctx.close()


def sample_nodes(ns, per_kind=40, seed=2014):
    # the node set is ordered by lattice row, so the body's surface nodes are found
    # by kind and position: wall nodes near the origin (the channel's walls are at
    # |x| = 8, 24 and |y| = 8)
    rng = np.random.default_rng(seed)
    r = np.hypot(ns.x, ns.y)
    idx = np.arange(ns.n)
    interior = ns.kind == vo.KIND_INTERIOR
    surface = (ns.kind == vo.KIND_WALL) & (r < 2.0)
    groups = {
        "interior": idx[interior & (r > 2.0)],
        "near body": idx[interior & (r < 1.2)],
        "walls": idx[~interior & ~surface],
        "surface": idx[surface],
    }
    assert groups["surface"].size == ns.meta["surface_nodes"]
    picks = {k: rng.choice(v, size=min(per_kind, v.size), replace=False) for k, v in groups.items()}
    for k, v in groups.items():
        assert v.size > 0, k
    return picks


def test_sampled_laplacian_rows_match_oracle(full):
    ns, ctx = full
    ptr, col, val = ctx.vip_get_stencil("LAPLACE")
    assert ptr.size == ns.n + 1
    for group, nodes in sample_nodes(ns).items():
        rho = 2.2 * ns.h[nodes]
        qptr, qidx = vo.neighbours(ns.x[nodes], ns.y[nodes], rho, ns.x, ns.y, ns.Lx, ns.Ly)
        wts = vo.mls_weights(ns.x[nodes], ns.y[nodes], rho, qptr, qidx, ns.x, ns.y, ns.Lx, ns.Ly,
                             "cubic_spline", derivs=((2, 0), (0, 2)))
        lap = wts[(2, 0)] + wts[(0, 2)]
        for k, i in enumerate(nodes):
            ref = dict(zip(qidx[qptr[k]:qptr[k + 1]].tolist(), lap[qptr[k]:qptr[k + 1]]))
            got = dict(zip(col[ptr[i]:ptr[i + 1]].tolist(), val[ptr[i]:ptr[i + 1]]))
            # same columns (an entry either side lacks counts as 0)
            scale = max(abs(v) for v in ref.values())
            err = max(abs(got.get(c, 0.0) - ref.get(c, 0.0)) for c in set(got) | set(ref))
            assert err <= 1e-10 * scale, (group, int(i), err / scale)
            assert set(got) <= set(ref), (group, int(i))


def test_full_size_poisson_solve_residual(full, vip):
    ns, ctx = full
    ptr, col, val = ctx.vip_get_stencil("POISSON")
    n = ptr.size - 1
    assert n == ns.n  # open channel: no bordering row
    P = sp.csr_matrix((val, col, ptr), shape=(n, n))
    rng = np.random.default_rng(5)
    b = np.where(ns.kind == vo.KIND_INTERIOR, rng.standard_normal(n), 0.0)
    # hierarchy of the 2049 x 1025 lattice: cells 1025 x 513, ..., 65 x 33 = 2145 <= 2200
    assert ctx.vip_multigrid_info() == (5, 2145 ** 2)
    x, it, rr = ctx.vip_solve("POISSON", b, np.zeros(n), precision=vip.VIP_PREC_FP64, rtol=1e-8,
                              max_iters=20000)
    assert 0 < it < 1000 and rr <= 1e-8, (it, rr)
    res = np.linalg.norm(b - P @ x) / np.linalg.norm(b)
    assert res <= 1.01e-8, res


def test_full_size_steps(full):
    ns, ctx = full
    for _ in range(2):
        ctx.vip_step(1)
        st = ctx.vip_get_stats()
        assert st.status == 0
        assert st.poisson_relres <= 1e-8 and st.helm_relres <= 1e-8
    u, v, p, phi = ctx.vip_get_state()
    assert all(np.all(np.isfinite(a)) for a in (u, v, p, phi))
    assert np.max(np.abs(u)) < 10.0  # impulsively started unit inflow stays bounded
