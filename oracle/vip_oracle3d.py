"""FP64 CPU oracle of the 3D extension of the VIP operator build.

Park, Jo and Choe, "Virtual Interpolation Point Method for Viscous Flows in
Complex Geometries" (arXiv:1401.6513).  The introduction and Sec. 3 state that the
method extends to three dimensions with the quadratic basis of ten monomials; the
paper shows no 3D flow.  This module states the 3D counterparts of the 2D oracle's
neighbour search, MLS derivative weights (Sec. 3, Eq. fmlsrk:2) and operators
(Eq. vip:1, Sec. 4.1), with the same readings: the cubic-spline weight, strict
support |x_i - xbar| < rho with rho = support * h of the point's own node,
"diffuse" derivatives of the local polynomial at its centre, VIPs at half the local
spacing along each axis (six in 3D: east/west, north/south, top/bottom), VIP
differences for the gradient, and at boundary nodes the zero-normal-derivative row
q_i - (4/3) q(x_i - h n) + (1/3) q(x_i - 2h n) with MLS values at the two normal
points.

TEST INFRASTRUCTURE ONLY.  Only the tests and the smoke check may import it; the
product path never does.  It shares no code with the CUDA path (its inputs come
from the seeded generators of ``workloads``).

Pins (tests/test_oracle_3d.py, all CPU):
  * neighbour lists equal a brute-force all-pairs test, periodic and not;
  * the weights reproduce all ten quadratic monomials and their derivatives at
    every node, VIP and normal point, and equal a weighted least-squares fit by
    SVD (numpy.linalg.lstsq) on sampled points;
  * L 1 = 0, L (x^2 + y^2 + z^2) = 6, Gx, Gy, Gz exact on quadratics at interior
    nodes, the Neumann rows equal (2/3) h dq/dn on quadratics;
  * L and G are second order on a smooth periodic field (observed order >= 1.8);
  * planted mistakes (a dropped factorial, a swapped VIP pair) fail the pins;
  * the 3D step (FractionalStep3) is second order in space on the exact ABC flow
    (velocity and pressure), and a convection of the wrong sign or a dropped
    z-difference fails that pin; in time the velocity is second order and the
    pressure first order (self-convergence), and a backward-Euler viscous term
    fails that pin; with walls, plane Poiseuille flow is a fixed point to 1e-12,
    and a wrong-signed Crank-Nicolson term or walls solved as interior rows move it.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
from scipy.spatial import cKDTree

from .vip_oracle import KIND_INTERIOR, WEIGHTS, SingularStencil, min_image

# The scaled quadratic basis in 3D, p = [1, xi, eta, zeta, xi^2, xi eta, xi zeta,
# eta^2, eta zeta, zeta^2], and the derivative (a, b, c) each coefficient stands for.
DERIVS3 = ((0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (1, 1, 0), (1, 0, 1),
           (0, 2, 0), (0, 1, 1), (0, 0, 2))

# The node derivative tables the 3D build exports.
NODE_DERIVS3 = ((0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (0, 2, 0), (0, 0, 2))

VIPS3 = ("e", "w", "n", "s", "t", "b")


def basis3(xi, eta, zeta):
    one = np.ones_like(xi)
    return np.stack([one, xi, eta, zeta, xi * xi, xi * eta, xi * zeta, eta * eta,
                     eta * zeta, zeta * zeta], axis=1)


def neighbours3(q, rho, pts, L=(0.0, 0.0, 0.0)):
    """Indices of the nodes strictly inside |x_i - q| < rho(q) for every query
    point q (rows of q), ascending per point, as CSR (ptr, idx).  The test is
    dx^2 + dy^2 + dz^2 < rho^2 with minimum-image differences in periodic
    directions; a k-d tree only proposes candidates."""
    q = np.asarray(q, np.float64)
    rho = np.broadcast_to(np.asarray(rho, np.float64), (q.shape[0],))
    if any(l > 0.0 for l in L):
        if not all(l > 0.0 for l in L):
            raise ValueError("periodic in every direction or in none")
        tree = cKDTree(pts, boxsize=list(L))
        qq = np.mod(q, np.asarray(L))
        for k in range(3):
            qq[qq[:, k] >= L[k], k] -= L[k]
    else:
        tree = cKDTree(pts)
        qq = q
    cand = tree.query_ball_point(qq, r=rho * (1.0 + 1e-9) + 1e-300)
    ptr = np.zeros(q.shape[0] + 1, np.int64)
    out = []
    for p, c in enumerate(cand):
        c = np.asarray(sorted(c), np.int64)
        d = [min_image(pts[c, k] - q[p, k], L[k]) for k in range(3)]
        keep = c[d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < rho[p] * rho[p]]
        out.append(keep)
        ptr[p + 1] = ptr[p] + keep.size
    idx = np.concatenate(out) if out else np.zeros(0, np.int64)
    return ptr, idx


def mls_weights3(q, rho, ptr, idx, pts, L=(0.0, 0.0, 0.0), weight="cubic_spline",
                 derivs=NODE_DERIVS3, cond_max=1e13):
    """Derivative weights of the 3D moving least-squares fit at each query point.

    For a point xbar with neighbours x_i (Sec. 3, in three coordinates):
    (xi, eta, zeta) = (x_i - xbar)/rho, p_i the ten monomials of basis3, Phi_i the
    weight of |x_i - xbar|/rho, M = sum_i Phi_i p_i p_i^T; the fit's coefficient k
    is (M^{-1} sum_i Phi_i p_i u_i)_k, and the (a,b,c) derivative of the local
    polynomial at xbar is a! b! c! rho^-(a+b+c) times the coefficient of its
    monomial.  Hence Psi^[a,b,c]_i = a! b! c! rho^-(a+b+c) Phi_i (M^{-1} p_i)_k
    (M^{-1} p_i by a dense LU solve).  Returns {deriv: values aligned with idx};
    SingularStencil when cond(M) > cond_max."""
    phi = WEIGHTS[weight]
    cnt = np.diff(ptr)
    P = cnt.size
    K = int(cnt.max()) if P else 0
    pad = np.zeros((P, K), np.int64)
    mask = np.arange(K)[None, :] < cnt[:, None]
    pad[mask] = idx
    q = np.asarray(q, np.float64)
    rho = np.broadcast_to(np.asarray(rho, np.float64), (P,))
    d = [min_image(pts[pad, k] - q[:, k, None], L[k]) / rho[:, None] for k in range(3)]
    W = np.where(mask, phi(np.sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2])), 0.0)
    Pm = basis3(*d) * mask[:, None, :]                      # [P, 10, K]
    M = np.einsum("pak,pk,pbk->pab", Pm, W, Pm)
    ev = np.linalg.eigvalsh(M)
    cond = ev[:, -1] / np.maximum(ev[:, 0], 1e-300)
    bad = np.nonzero(~(cond < cond_max))[0]
    if bad.size:
        raise SingularStencil(int(bad[0]), float(cond[bad[0]]))
    Z = np.linalg.solve(M, Pm)
    out = {}
    for a in derivs:
        k = DERIVS3.index(a)
        fac = math.factorial(a[0]) * math.factorial(a[1]) * math.factorial(a[2]) / rho ** sum(a)
        out[a] = (fac[:, None] * W * Z[:, k, :])[mask]
    return out


def _csr(rows, ptr, idx, val, N):
    r = np.repeat(rows, np.diff(ptr))
    return sp.csr_matrix((val, (r, idx)), shape=(N, N))


class Operators3:
    """Sparse FP64 operators of the 3D VIP build on a NodeSet3.

    D[(a,b,c)]  node derivative approximants for NODE_DERIVS3 (N x N)
    L           D^[2,0,0] + D^[0,2,0] + D^[0,0,2]
    I[k]        interpolation Psi^[0,0,0](x_vip) to the six VIPs of interior nodes,
                k in VIPS3 (rows of boundary nodes empty)
    Gx, Gy, Gz  (u(x_e) - u(x_w))/|x_e - x_w|, (u(x_n) - u(x_s))/|x_n - x_s|,
                (u(x_t) - u(x_b))/|x_t - x_b|
    Nb          q_i - (4/3) q(x_i - h n_i) + (1/3) q(x_i - 2 h n_i) at boundary nodes
    """

    def __init__(self, ns, weight="cubic_spline", support=2.2):
        pts = np.stack([ns.x, ns.y, ns.z], 1)
        N = ns.n
        L = (ns.Lx, ns.Ly, ns.Lz)
        h = ns.h
        rho = support * h
        self.N, self.ns, self.pts, self.L3 = N, ns, pts, L
        self.node_ptr, self.node_idx = neighbours3(pts, rho, pts, L)
        wn = mls_weights3(pts, rho, self.node_ptr, self.node_idx, pts, L, weight)
        every = np.arange(N)
        self.D = {a: _csr(every, self.node_ptr, self.node_idx, wn[a], N) for a in NODE_DERIVS3}
        self.L = ((self.D[(2, 0, 0)] + self.D[(0, 2, 0)]) + self.D[(0, 0, 2)]).tocsr()
        ii = np.nonzero(ns.kind == KIND_INTERIOR)[0]
        self.interior = ii
        hh = 0.5 * h[ii]
        self.vip = {}
        for k, (ax, sgn) in zip(VIPS3, ((0, 1), (0, -1), (1, 1), (1, -1), (2, 1), (2, -1))):
            v = pts[ii].copy()
            v[:, ax] = v[:, ax] + hh if sgn > 0 else v[:, ax] - hh
            self.vip[k] = v
        self.vip_ptr, self.vip_idx, self.I = {}, {}, {}
        for k, v in self.vip.items():
            ptr, idx = neighbours3(v, rho[ii], pts, L)
            w = mls_weights3(v, rho[ii], ptr, idx, pts, L, weight, derivs=((0, 0, 0),))[(0, 0, 0)]
            self.vip_ptr[k], self.vip_idx[k] = ptr, idx
            self.I[k] = _csr(ii, ptr, idx, w, N)
        G = []
        for ax, (p, m) in enumerate((("e", "w"), ("n", "s"), ("t", "b"))):
            inv = np.zeros(N)
            inv[ii] = 1.0 / np.abs(self.vip[p][:, ax] - self.vip[m][:, ax])
            G.append((sp.diags(inv) @ (self.I[p] - self.I[m])).tocsr())
        self.Gx, self.Gy, self.Gz = G
        bb = np.nonzero(ns.kind != KIND_INTERIOR)[0]
        self.boundary = bb
        nrm = np.stack([ns.nx, ns.ny, ns.nz], 1)[bb]
        self.probe = {s: pts[bb] - s * h[bb, None] * nrm for s in (1, 2)}
        B = {}
        for s, v in self.probe.items():
            ptr, idx = neighbours3(v, rho[bb], pts, L)
            w = mls_weights3(v, rho[bb], ptr, idx, pts, L, weight, derivs=((0, 0, 0),))[(0, 0, 0)]
            B[s] = _csr(bb, ptr, idx, w, N)
        self.B = B
        sel = np.zeros(N)
        sel[bb] = 1.0
        self.Nb = (sp.diags(sel) - (4.0 / 3.0) * B[1] + (1.0 / 3.0) * B[2]).tocsr()


# ---------------------------------------------------------------------------
# The fractional step in three coordinates (Sec. 2, Eqs. 12-15)
# ---------------------------------------------------------------------------

def convection3(ops: Operators3, u, v, w):
    """Convection at the interior nodes (zero at wall nodes) via the six VIPs (Sec. 4.1 item 1
    in three coordinates): the products of interpolated values, differenced across
    each VIP pair and divided by the pair distance (the flux form of u . grad u)."""
    I = ops.I
    e = {k: (I[k] @ u, I[k] @ v, I[k] @ w) for k in VIPS3}
    ii = ops.interior
    inv = []
    for ax, (p, m) in enumerate((("e", "w"), ("n", "s"), ("t", "b"))):
        a = np.zeros(ops.N)
        a[ii] = 1.0 / np.abs(ops.vip[p][:, ax] - ops.vip[m][:, ax])
        inv.append(a)
    out = []
    for c in range(3):           # component c of the momentum flux
        f = ((e["e"][0] * e["e"][c] - e["w"][0] * e["w"][c]) * inv[0]
             + (e["n"][1] * e["n"][c] - e["s"][1] * e["s"][c]) * inv[1]
             + (e["t"][2] * e["t"][c] - e["b"][2] * e["b"][c]) * inv[2])
        out.append(f)
    return out


class FractionalStep3:
    """The second-order fractional step of the 2D oracle in three coordinates:
    AB2 convection, Crank-Nicolson viscous term, the incremental pressure reading
    (r^n carries -G p^n, phi the increment, p^{n+1} = p^n + phi - (dt/2Re) L phi at
    every node), exact identity, the MLS Laplacian in the Poisson equation,
    unpreconditioned BiCGSTAB.  Node kinds: interior, and wall (velocity
    Dirichlet, holding the node's initial value; pressure-increment zero normal
    derivative through the Neumann rows, scaled by -6/h^2 so that their diagonal
    has the sign and size of the 3D Laplacian rows).  Every 3D problem here has no
    Dirichlet row for phi, so, as in the 2D oracle, the Poisson system is bordered
    by one unknown mu added to the interior rows, the first interior node k0's own
    equation moved to an extra row and its row replaced by (-6/h_k0^2) phi_k0 = 0."""

    def __init__(self, ops: Operators3, Re, dt, rtol=1e-8, maxit=200000):
        kind = ops.ns.kind
        if np.any((kind != KIND_INTERIOR) & (kind != 1)):
            raise ValueError("the 3D step takes interior and wall nodes only")
        from .vip_oracle import bicgstab
        self._bicgstab = bicgstab
        N = ops.N
        self.ops, self.N = ops, N
        self.Re, self.dt = float(Re), float(dt)
        self.rtol, self.maxit = rtol, maxit
        self.alpha = self.dt / (2.0 * self.Re)
        inner = kind == KIND_INTERIOR
        self.inner = inner
        S = lambda m: sp.diags(m.astype(np.float64))  # noqa: E731  row selection
        Id = sp.identity(N, format="csr")
        self.H = (S(inner) @ (Id - self.alpha * ops.L) + S(~inner) @ Id).tocsr()
        self.Rm = (Id + self.alpha * ops.L).tocsr()
        pin_scale = -6.0 / ops.ns.h ** 2
        P = (S(inner) @ ops.L + sp.diags(~inner * pin_scale) @ ops.Nb).tocsr()
        k0 = int(np.nonzero(inner)[0][0])
        self.pin = k0
        Pb = sp.bmat([[P, sp.csr_matrix(inner.astype(np.float64)[:, None])],
                      [sp.csr_matrix((1, N)), None]]).tolil()
        rowk = Pb[k0].copy()
        Pb[k0] = 0.0
        Pb[k0, k0] = pin_scale[k0]
        Pb[N] = rowk
        self.P = Pb.tocsr()
        self.u = np.zeros(N)
        self.v = np.zeros(N)
        self.w = np.zeros(N)
        self.p = np.zeros(N)
        self.phi = np.zeros(N)
        self.mu = 0.0
        self.bc = (np.zeros(N),) * 3
        self.N_prev = None
        self.nstep = 0

    def set_state(self, u, v, w, p):
        """Fields at every node; the wall nodes' velocities become their boundary
        values."""
        self.u, self.v, self.w, self.p = (np.array(a, np.float64) for a in (u, v, w, p))
        self.bc = (self.u.copy(), self.v.copy(), self.w.copy())
        self.phi = np.zeros(self.N)
        self.mu = 0.0
        self.N_prev = None

    def step(self):
        ops, dt, inner = self.ops, self.dt, self.inner
        vel = (self.u, self.v, self.w)
        Nn = convection3(ops, *vel)
        if self.N_prev is None:
            self.N_prev = Nn
        Nab = [1.5 * a - 0.5 * b for a, b in zip(Nn, self.N_prev)]
        self.N_prev = Nn
        G = (ops.Gx, ops.Gy, ops.Gz)
        star = []
        for c in range(3):        # Eq. (12) times dt, per component; walls hold their values
            r = np.where(inner, self.Rm @ vel[c] - dt * (Nab[c] + G[c] @ self.p), self.bc[c])
            star.append(self._bicgstab(self.H, r, vel[c], self.rtol, self.maxit)[0])
        b = np.where(inner, (ops.Gx @ star[0] + ops.Gy @ star[1] + ops.Gz @ star[2]) / dt, 0.0)
        b = np.append(b, b[self.pin])                                        # Eq. (13)
        b[self.pin] = 0.0
        sol = self._bicgstab(self.P, b, np.append(self.phi, self.mu), self.rtol, self.maxit)[0]
        phi = sol[:self.N]
        self.mu = float(sol[-1])
        self.u, self.v, self.w = (np.where(inner, star[c] - dt * (G[c] @ phi), star[c])
                                  for c in range(3))                          # Eq. (14)
        self.p = self.p + phi - self.alpha * (ops.L @ phi)                   # Eq. (15)
        self.phi = phi
        self.nstep += 1


def abc_flow(x, y, z, t, Re, A=1.0, B=0.8, C=0.6):
    """The Arnold-Beltrami-Childress field, an exact decaying Navier-Stokes solution
    on the 2 pi periodic cube: curl u = u and Lap u = -u, so u . grad u =
    grad(|u|^2 / 2) and u = U(x) exp(-t/Re), p = -|u|^2 / 2 (up to a constant)."""
    f = np.exp(-t / Re)
    u = (A * np.sin(z) + C * np.cos(y)) * f
    v = (B * np.sin(x) + A * np.cos(z)) * f
    w = (C * np.sin(y) + B * np.cos(x)) * f
    return u, v, w, -0.5 * (u * u + v * v + w * w)
