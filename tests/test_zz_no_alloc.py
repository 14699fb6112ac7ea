"""vip_bicgstab_static (BiCGSTAB with a static device workspace, no allocation)
against vip_solve on the same systems, through the C ABI.

The file name sorts last so that the call also runs after every other GPU test
has used the device.  The test itself allocates its buffers with torch; the
entry point under test allocates nothing.

Tolerances: both solvers stop at relative residual 1e-12 in FP64, so their
solutions differ by at most ~cond(A) * 1e-12 relative; cond is ~1e2 for the
Helmholtz operator and ~1e4 for the bordered Poisson operator of these grids,
hence the bars 1e-9 and 1e-7.  Two calls in a row on the same input must agree
bit for bit (fixed grid, fixed reduction order).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(vip):
    c = vip.solver_for(w.cavity(40, Re=400.0), precision=vip.VIP_PREC_FP64)
    yield c
    c.close()


def device_csr(ctx, which):
    import torch
    ptr, col, val = ctx.vip_get_stencil(which)
    dev = torch.device("cuda:0")
    return (ptr.size - 1, torch.from_numpy(ptr).to(dev), torch.from_numpy(col).to(dev),
            torch.from_numpy(val).to(dev), (ptr, col, val))


@pytest.mark.parametrize("which,bar", [("HELM_U", 1e-9), ("POISSON", 1e-7)])
def test_matches_vip_solve_twice(vip, ctx, which, bar):
    import torch
    n, dptr, dcol, dval, (ptr, col, val) = device_csr(ctx, which)
    rng = np.random.default_rng(11)
    b = rng.standard_normal(n)
    ref, _, rr_ref = ctx.vip_solve(which, b, np.zeros(n), precision=vip.VIP_PREC_FP64, rtol=1e-12,
                                   max_iters=200000)
    assert rr_ref <= 1e-11
    db = torch.from_numpy(b).cuda()
    sols = []
    for _ in range(2):
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        st, it, rr = vip.vip_bicgstab_static(0, None, n, dptr, dcol, dval, db, x, rtol=1e-12,
                                             max_iters=200000)
        assert st == vip.VIP_OK, (st, it, rr)
        assert 0 < it and rr <= 1e-11
        sols.append(x.cpu().numpy())
    A = sp.csr_matrix((val, col, ptr), shape=(n, n))
    for x in sols:
        assert np.linalg.norm(b - A @ x) <= 1e-11 * np.linalg.norm(b)
        assert np.linalg.norm(x - ref) <= bar * np.linalg.norm(ref)
    assert np.array_equal(sols[0], sols[1])


def test_largest_size(vip):
    """n = VIP_STATIC_MAX_ROWS: a diagonally dominant nonsymmetric 5-point operator
    on a 512 x 256 grid (convection-diffusion shape)."""
    import torch
    nx, ny = 512, 256
    n = nx * ny
    assert n == vip.VIP_STATIC_MAX_ROWS
    I = sp.identity(nx)
    J = sp.identity(ny)
    tx = sp.diags([-1.3, 2.0, -0.7], [-1, 0, 1], shape=(nx, nx))
    ty = sp.diags([-1.1, 2.0, -0.9], [-1, 0, 1], shape=(ny, ny))
    A = (sp.kron(J, tx) + sp.kron(ty, I) + 0.5 * sp.identity(n)).tocsr()
    A.sort_indices()
    b = np.random.default_rng(5).standard_normal(n)
    dev = "cuda"
    dptr = torch.from_numpy(A.indptr.astype(np.int64)).to(dev)
    dcol = torch.from_numpy(A.indices.astype(np.int32)).to(dev)
    dval = torch.from_numpy(A.data.astype(np.float64)).to(dev)
    db = torch.from_numpy(b).to(dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    st, it, rr = vip.vip_bicgstab_static(0, None, n, dptr, dcol, dval, db, x, rtol=1e-10)
    assert st == vip.VIP_OK and rr <= 1e-9, (st, it, rr)
    xs = x.cpu().numpy()
    assert np.linalg.norm(b - A @ xs) <= 1e-9 * np.linalg.norm(b)


def test_rejects_bad_arguments(vip):
    """Too many rows and host pointers are refused before any device work."""
    import torch
    n = 8
    dptr = torch.arange(n + 1, dtype=torch.int64, device="cuda")
    dcol = torch.arange(n, dtype=torch.int32, device="cuda")
    dval = torch.ones(n, dtype=torch.float64, device="cuda")
    db = torch.ones(n, dtype=torch.float64, device="cuda")
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    big = vip.VIP_STATIC_MAX_ROWS + 1
    st, _, _ = vip.vip_bicgstab_static(0, None, big, dptr, dcol, dval, db, x)
    assert st == vip.VIP_ERR_ARG
    hb = np.ones(n)
    st, _, _ = vip.vip_bicgstab_static(0, None, n, dptr, dcol, dval, hb, x)
    assert st == vip.VIP_ERR_ARG
    st, _, _ = vip.vip_bicgstab_static(0, None, n, dptr, dcol, dval, db, x, rtol=0.0)
    assert st == vip.VIP_ERR_ARG
    # the identity system still solves after the refusals
    st, it, rr = vip.vip_bicgstab_static(0, None, n, dptr, dcol, dval, db, x)
    assert st == vip.VIP_OK and np.allclose(x.cpu().numpy(), 1.0)


def test_refuses_a_capturing_stream(vip):
    """The call synchronises its stream and reads its result back, so on a stream that
    is being captured into a CUDA graph it returns VIP_ERR_ARG before any work and the
    capture stays valid."""
    import torch
    n = 8
    dptr = torch.arange(n + 1, dtype=torch.int64, device="cuda")
    dcol = torch.arange(n, dtype=torch.int32, device="cuda")
    dval = torch.ones(n, dtype=torch.float64, device="cuda")
    db = torch.ones(n, dtype=torch.float64, device="cuda")
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        x.add_(0.0)
        st, _, _ = vip.vip_bicgstab_static(0, s.cuda_stream, n, dptr, dcol, dval, db, x)
    assert st == vip.VIP_ERR_ARG
    g.replay()
    torch.cuda.synchronize()
    st, it, rr = vip.vip_bicgstab_static(0, None, n, dptr, dcol, dval, db, x)
    assert st == vip.VIP_OK and np.allclose(x.cpu().numpy(), 1.0)
