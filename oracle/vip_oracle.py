"""FP64 CPU oracle of the virtual interpolation point (VIP) fractional-step method.

Park, Jo and Choe, "Virtual Interpolation Point Method for Viscous Flows in
Complex Geometries" (arXiv:1401.6513).

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously correct
statement of what the CUDA path computes.  Only the tests, the smoke check and
the CPU-baseline leg of the benchmark may import it; the product path never
does.  It shares no code with the CUDA path: the two sides meet only in the
seeded input generators of the ``workloads`` package.

Every function cites the passage it follows.  Where the paper is silent or
garbled the reading used is stated at the function (the readings are listed in
one place in the design notes of the repository).

Pins (tests/test_oracle_*.py, all CPU):
  * weight functions: values, continuity and support; the printed weight's
    expansion at both ends of its support, Phi(1 - s) = s^12 (1 + 2s + ...) and
    (1 - Phi(r)) / r -> 4 (Sec. 3);
  * neighbour search: brute force on small node sets, periodic and not;
  * MLS weights: exact reproduction of the six quadratic monomials and their
    derivatives, and agreement with a brute-force weighted least-squares fit by
    SVD (numpy.linalg.lstsq) on small stencils (Sec. 3, Eq. fmlsrk:2);
  * operators: L.1 = 0, L.(x^2+y^2) = 4, D00 q = q, Gx q = dq/dx exactly for
    quadratics (Eq. vip:1, Sec. 4.1 items 2-3);
  * convection: equals the flux difference of exact VIP values for quadratic
    velocity fields (Sec. 4.1 item 1);
  * BiCGSTAB: agrees with a sparse direct solve (scipy spsolve);
  * full step: observed second order in space and time on the decaying
    vortices (Sec. 5.1) and the divergence of the projected velocity at the
    Poisson tolerance in the composite-operator reading (Eqs. 13-14);
  * the alternative readings: pressure="kim_moin" gives the time-centred
    pressure of the decaying vortices (closed form at t - dt/2) and the
    incremental reading's pressure (Eq. 15); identity="mls" agrees with the exact
    identity on quadratics and keeps second order (Eq. 12, Eq. vip:1); mistakes
    planted in these pins are caught (test_planted_mistakes_are_caught);
  * normal points (flag probes="inside", tests/test_paper_values.py): inside
    the exact edges of the 28-degree wedge cavity, unchanged on the square
    cavity, and the wedge's steps stable with them and unstable without;
  * pressure="incremental_interior" (tests/test_oracle_pins.py): identical to the
    incremental reading, bit for bit, where there are no boundary nodes (the
    periodic box), and on the wedge (normal points inside) the step linearised
    about rest has no eigenvalue above 1, where the incremental reading has one
    (1 + 8.7e-4); planted mistakes in it are caught.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
from scipy.spatial import cKDTree

# Node kinds: the one-byte input encoding of the node set.
KIND_INTERIOR = 0
KIND_WALL = 1      # velocity Dirichlet, pressure-increment Neumann
KIND_SLIP = 2      # u Neumann, v Dirichlet, pressure-increment Neumann
KIND_OUTLET = 3    # velocity Neumann, pressure-increment Dirichlet (zero)


class SingularStencil(RuntimeError):
    """The moment matrix of some point is (numerically) singular."""

    def __init__(self, point: int, cond: float):
        super().__init__(f"singular MLS moment matrix at point {point} (cond {cond:.3e})")
        self.point = point


class KrylovBreakdown(RuntimeError):
    pass


# ---------------------------------------------------------------------------
# Sec. 3: weight function Phi
# ---------------------------------------------------------------------------

def weight_cubic_spline(r):
    """Cubic B-spline weight in r = |x_i - xbar| / rho (the weight named by the workloads).

    2/3 - 4r^2 + 4r^3 for r <= 1/2, 4/3 - 4r + 4r^2 - 4r^3/3 for 1/2 < r < 1, 0 otherwise.
    Its constant factor cancels in the MLS weights.
    """
    r = np.asarray(r, dtype=np.float64)
    w = np.zeros_like(r)
    a = r <= 0.5
    b = (r > 0.5) & (r < 1.0)
    w[a] = 2.0 / 3.0 - 4.0 * r[a] ** 2 + 4.0 * r[a] ** 3
    w[b] = 4.0 / 3.0 - 4.0 * r[b] + 4.0 * r[b] ** 2 - (4.0 / 3.0) * r[b] ** 3
    return w


def weight_paper(r):
    """The weight printed in Sec. 3: (1 - |y|^((1-|y|)^2))^4 for |y| < 1, else 0."""
    r = np.asarray(r, dtype=np.float64)
    w = np.zeros_like(r)
    a = r < 1.0
    w[a] = (1.0 - np.power(r[a], (1.0 - r[a]) ** 2)) ** 4
    return w


WEIGHTS = {"cubic_spline": weight_cubic_spline, "paper": weight_paper}


# ---------------------------------------------------------------------------
# Sec. 3: the neighbourhood of a point (nodes x_i with |x_i - xbar| < rho)
# ---------------------------------------------------------------------------

def min_image(d, L):
    """Periodic minimum image of a coordinate difference (one correction by +-L)."""
    if L <= 0.0:
        return d
    d = np.where(d > 0.5 * L, d - L, d)
    return np.where(d < -0.5 * L, d + L, d)


def neighbours(qx, qy, rho, x, y, Lx=0.0, Ly=0.0):
    """Indices of nodes strictly inside the support |x_i - q| < rho(q) of every query point.

    Returns CSR-style (ptr, idx) with ascending node indices per point.  The
    support test is d^2 < rho^2 with d the (minimum-image) difference x_i - q.
    A k-d tree only proposes candidates; membership is decided by that test.
    """
    qx = np.asarray(qx, np.float64)
    qy = np.asarray(qy, np.float64)
    rho = np.broadcast_to(np.asarray(rho, np.float64), qx.shape)
    if Lx > 0.0 or Ly > 0.0:
        tree = cKDTree(np.stack([x, y], 1), boxsize=[Lx, Ly])
        qq = np.stack([np.mod(qx, Lx), np.mod(qy, Ly)], 1)
        qq[qq[:, 0] >= Lx, 0] -= Lx
        qq[qq[:, 1] >= Ly, 1] -= Ly
    else:
        tree = cKDTree(np.stack([x, y], 1))
        qq = np.stack([qx, qy], 1)
    cand = tree.query_ball_point(qq, r=rho * (1.0 + 1e-9) + 1e-300)
    ptr = np.zeros(qx.size + 1, np.int64)
    out = []
    for p, c in enumerate(cand):
        c = np.asarray(sorted(c), np.int64)
        dx = min_image(x[c] - qx[p], Lx)
        dy = min_image(y[c] - qy[p], Ly)
        keep = c[dx * dx + dy * dy < rho[p] * rho[p]]
        out.append(keep)
        ptr[p + 1] = ptr[p] + keep.size
    idx = np.concatenate(out) if out else np.zeros(0, np.int64)
    return ptr, idx


# ---------------------------------------------------------------------------
# Sec. 3: MLS derivative weights Psi^[a,b]_i(xbar), Eq. (fmlsrk:2)
# ---------------------------------------------------------------------------

# Monomials of the scaled quadratic basis p = [1, xi, eta, xi^2, xi eta, eta^2]
# and the derivative (a,b) each coefficient c_k represents at xbar.
DERIVS = ((0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2))


def _padded(ptr, idx):
    cnt = np.diff(ptr)
    K = int(cnt.max()) if cnt.size else 0
    P = cnt.size
    pad = np.zeros((P, K), np.int64)
    mask = np.arange(K)[None, :] < cnt[:, None]
    pad[mask] = idx
    return pad, mask


def mls_weights(qx, qy, rho, ptr, idx, x, y, Lx=0.0, Ly=0.0, weight="cubic_spline",
                derivs=DERIVS, cond_max=1e13):
    """Derivative weights of the moving least-squares fit at each query point xbar.

    For each point (Sec. 3):
      xi = (x_i - xbar)/rho, eta = (y_i - ybar)/rho, p_i = [1, xi, eta, xi^2, xi eta, eta^2];
      the minimiser of J(c) = sum_i Phi(|x_i - xbar|/rho) |p_i . c - u_i|^2 is
      c = M^{-1} sum_i Phi_i p_i u_i with M = sum_i Phi_i p_i p_i^T;
      u_m(x, xbar) = p((x - xbar)/rho) . c, and D^[a,b]u(xbar) is its (a,b)
      derivative at x = xbar, which picks coefficient k of (a,b) times a! b! rho^-(a+b).
    Hence Psi^[a,b]_i = a! b! rho^-(a+b) Phi_i (M^{-1} p_i)_k.  M^{-1} p_i is obtained
    from a dense LU solve (numpy.linalg.solve).

    Returns {deriv: values aligned with idx}.
    Raises SingularStencil when cond(M) > cond_max.
    """
    phi = WEIGHTS[weight]
    pad, mask = _padded(ptr, idx)
    qx = np.asarray(qx, np.float64)
    qy = np.asarray(qy, np.float64)
    rho = np.broadcast_to(np.asarray(rho, np.float64), qx.shape)
    dx = min_image(x[pad] - qx[:, None], Lx)
    dy = min_image(y[pad] - qy[:, None], Ly)
    xi = dx / rho[:, None]
    eta = dy / rho[:, None]
    W = np.where(mask, phi(np.sqrt(xi * xi + eta * eta)), 0.0)
    one = np.ones_like(xi)
    Pm = np.stack([one, xi, eta, xi * xi, xi * eta, eta * eta], axis=1)  # [P, 6, K]
    Pm = Pm * mask[:, None, :]
    M = np.einsum("pak,pk,pbk->pab", Pm, W, Pm)
    ev = np.linalg.eigvalsh(M)
    cond = ev[:, -1] / np.maximum(ev[:, 0], 1e-300)
    bad = np.nonzero(~(cond < cond_max))[0]
    if bad.size:
        raise SingularStencil(int(bad[0]), float(cond[bad[0]]))
    Z = np.linalg.solve(M, Pm)  # M^{-1} p_i, [P, 6, K]
    out = {}
    for (a, b) in derivs:
        k = DERIVS.index((a, b))
        fac = math.factorial(a) * math.factorial(b) / rho ** (a + b)
        out[(a, b)] = (fac[:, None] * W * Z[:, k, :])[mask]
    return out


# ---------------------------------------------------------------------------
# Sec. 4: virtual interpolation points and operators
# ---------------------------------------------------------------------------

class Operators:
    """Sparse FP64 operators of the VIP method on a node set (Eq. vip:1, Sec. 4.1).

    D[(a,b)]   node derivative approximants D^[a,b] (N x N)
    L          MLS Laplacian D^[2,0] + D^[0,2]                   (Eq. vip:1)
    Ie,Iw,In,Is interpolation to the four VIPs of each interior node (rows of
               non-interior nodes are empty): u(x_vip) = sum_i Psi^[0,0]_i(x_vip) u_i
    Gx, Gy     VIP differences (u(x_e)-u(x_w))/|x_e-x_w|, (u(x_n)-u(x_s))/|x_n-x_s|
               -- the divergence (item 2) and gradient (item 3) of Sec. 4.1.
    """

    def __init__(self, ns, weight="cubic_spline", support=2.2, probes="normal"):
        x, y, h = ns.x, ns.y, ns.h
        N = ns.n
        self.N = N
        self.ns = ns
        self.weight = weight
        self.support = support
        rho = support * h
        self.node_ptr, self.node_idx = neighbours(x, y, rho, x, y, ns.Lx, ns.Ly)
        wn = mls_weights(x, y, rho, self.node_ptr, self.node_idx, x, y, ns.Lx, ns.Ly, weight)
        self.node_w = wn
        self.D = {d: self._csr(self.node_ptr, self.node_idx, wn[d], N) for d in DERIVS}
        self.L = (self.D[(2, 0)] + self.D[(0, 2)]).tocsr()
        # VIPs at half the local spacing along each axis (reading: the figure of
        # Sec. 4.1 is missing; points at +-h/2 are the virtual staggered positions)
        self.interior = np.nonzero(ns.kind == KIND_INTERIOR)[0]
        ii = self.interior
        hh = 0.5 * h[ii]
        self.vip = {
            "e": (x[ii] + hh, y[ii]), "w": (x[ii] - hh, y[ii]),
            "n": (x[ii], y[ii] + hh), "s": (x[ii], y[ii] - hh),
        }
        self.vip_ptr, self.vip_idx, self.vip_w = {}, {}, {}
        self.I = {}
        for k, (qx, qy) in self.vip.items():
            ptr, idx = neighbours(qx, qy, rho[ii], x, y, ns.Lx, ns.Ly)
            w = mls_weights(qx, qy, rho[ii], ptr, idx, x, y, ns.Lx, ns.Ly, weight,
                            derivs=((0, 0),))[(0, 0)]
            self.vip_ptr[k], self.vip_idx[k], self.vip_w[k] = ptr, idx, w
            rows = np.repeat(ii, np.diff(ptr))
            self.I[k] = sp.csr_matrix((w, (rows, idx)), shape=(N, N))
        # 1/|x_e - x_w| and 1/|x_n - x_s| (the points differ along one axis only)
        self.inv_ew = np.zeros(N)
        self.inv_ns = np.zeros(N)
        self.inv_ew[ii] = 1.0 / np.abs(self.vip["e"][0] - self.vip["w"][0])
        self.inv_ns[ii] = 1.0 / np.abs(self.vip["n"][1] - self.vip["s"][1])
        self.Gx = (sp.diags(self.inv_ew) @ (self.I["e"] - self.I["w"])).tocsr()
        self.Gy = (sp.diags(self.inv_ns) @ (self.I["n"] - self.I["s"])).tocsr()
        # Auxiliary points on the inward normal of every boundary node, at one and two
        # local spacings (reading: the paper gives no boundary treatment for phi; a
        # zero normal derivative is imposed by the one-sided second-order difference
        # q_i = (4 q(x_i + h n_in) - q(x_i + 2 h n_in)) / 3 with MLS values there).
        self.boundary = np.nonzero(ns.kind != KIND_INTERIOR)[0]
        bb = self.boundary
        if probes == "normal":
            step = h[bb].copy()
        elif probes == "inside":
            step = self._probe_steps_inside(ns, bb)
        else:
            raise ValueError(f"probes must be 'normal' or 'inside', not {probes!r}")
        self.probe_step = step
        self.probe = {
            1: (x[bb] - step * ns.nx[bb], y[bb] - step * ns.ny[bb]),
            2: (x[bb] - 2.0 * step * ns.nx[bb], y[bb] - 2.0 * step * ns.ny[bb]),
        }
        self.B = {}
        for k, (qx, qy) in self.probe.items():
            ptr, idx = neighbours(qx, qy, rho[bb], x, y, ns.Lx, ns.Ly)
            w = mls_weights(qx, qy, rho[bb], ptr, idx, x, y, ns.Lx, ns.Ly, weight,
                            derivs=((0, 0),))[(0, 0)]
            rows = np.repeat(bb, np.diff(ptr))
            self.B[k] = sp.csr_matrix((w, (rows, idx)), shape=(N, N))
        sel = np.zeros(N)
        sel[bb] = 1.0
        # Neumann operator: q_i - (4/3) q(probe 1) + (1/3) q(probe 2) on boundary rows
        self.Nb = (sp.diags(sel) - (4.0 / 3.0) * self.B[1] + (1.0 / 3.0) * self.B[2]).tocsr()

    @staticmethod
    def _probe_steps_inside(ns, bb):
        """Reading (flag probes="inside"; the paper gives no boundary treatment for
        phi): where walls meet at a narrow angle the normal points can pass through
        the opposite wall.  A boundary node's step starts at its h_local and shrinks
        by 0.7 (at most 12 times) until its second normal point lies on the inner
        side of the tangent at the boundary node nearest to that point, by 5 % of
        that node's spacing."""
        bx, by = ns.x[bb], ns.y[bb]
        tree = cKDTree(np.stack([bx, by], 1))
        step = ns.h[bb].copy()
        for _ in range(12):
            qx, qy = bx - 2.0 * step * ns.nx[bb], by - 2.0 * step * ns.ny[bb]
            _, j = tree.query(np.stack([qx, qy], 1))
            side = (qx - bx[j]) * ns.nx[bb][j] + (qy - by[j]) * ns.ny[bb][j]
            bad = side > -0.05 * ns.h[bb][j]
            if not bad.any():
                break
            step = np.where(bad, 0.7 * step, step)
        return step

    @staticmethod
    def _csr(ptr, idx, val, N):
        return sp.csr_matrix((val, idx, ptr), shape=(ptr.size - 1, N))


def convection(ops: Operators, u, v):
    """Convection term at interior nodes via the VIPs (Sec. 4.1, item 1).

    Products of interpolated values (u(x_e)^2, u(x_n) v(x_n), ...) are differenced
    across each pair of VIPs and divided by the pair distance.  Zero at
    non-interior nodes.
    """
    I = ops.I
    ue, uw, un, us = I["e"] @ u, I["w"] @ u, I["n"] @ u, I["s"] @ u
    ve, vw, vn, vs = I["e"] @ v, I["w"] @ v, I["n"] @ v, I["s"] @ v
    Nu = (ue * ue - uw * uw) * ops.inv_ew + (un * vn - us * vs) * ops.inv_ns
    Nv = (ue * ve - uw * vw) * ops.inv_ew + (vn * vn - vs * vs) * ops.inv_ns
    return Nu, Nv


# ---------------------------------------------------------------------------
# Krylov solver (the paper does not name one; the operators are non-symmetric)
# ---------------------------------------------------------------------------

def bicgstab(A, b, x0=None, rtol=1e-8, maxit=100000, breakdown_tol=1e-12):
    """Unpreconditioned BiCGSTAB (van der Vorst, 1992) to ||b - A x||_2 <= rtol ||b||_2.

    The shadow residual is r_hat = r at the start.  When |r_hat . r| (or
    |r_hat . v|) drops below breakdown_tol ||r_hat|| ||r|| (||v||) the method would
    break down, so it restarts from the current x with r_hat = r.  Convergence is
    confirmed on the true residual b - A x; if only the recursively updated
    residual met the tolerance the iteration also restarts.  Returns
    (x, iterations, true relative residual).
    """
    b = np.asarray(b, np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, np.float64, copy=True)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0
    it = 0
    restarts = 0
    while it < maxit:
        r = b - A @ x
        if np.linalg.norm(r) <= rtol * bnorm:
            break
        restarts += 1
        if restarts > 1000:
            raise KrylovBreakdown("no progress after 1000 restarts")
        rhat = r.copy()
        rhat_norm = float(np.linalg.norm(rhat))
        rho_old = alpha = omega = 1.0
        v = np.zeros_like(b)
        p = np.zeros_like(b)
        while it < maxit:
            rho = float(rhat @ r)
            if abs(rho) <= breakdown_tol * rhat_norm * float(np.linalg.norm(r)):
                break  # restart
            it += 1
            beta = (rho / rho_old) * (alpha / omega)
            p = r + beta * (p - omega * v)
            v = A @ p
            rv = float(rhat @ v)
            if abs(rv) <= breakdown_tol * rhat_norm * float(np.linalg.norm(v)):
                break  # restart
            alpha = rho / rv
            s = r - alpha * v
            if np.linalg.norm(s) <= rtol * bnorm:
                x = x + alpha * p
                break
            t = A @ s
            tt = float(t @ t)
            if tt == 0.0:
                x = x + alpha * p
                break
            omega = float(t @ s) / tt
            x = x + alpha * p + omega * s
            r = s - omega * t
            if np.linalg.norm(r) <= rtol * bnorm or omega == 0.0:
                break
            rho_old = rho
    res = float(np.linalg.norm(b - A @ x)) / bnorm
    return x, it, res


# ---------------------------------------------------------------------------
# Sec. 2: the fractional step, Eqs. (12)-(15)
# ---------------------------------------------------------------------------

class FractionalStep:
    """Second-order fractional step on the VIP operators (Sec. 2, Sec. 4).

    Readings (the paper is silent or ambiguous on these):
      identity  'mls'  : I = D^[0,0] wherever the paper writes I (Eq. vip:1);
                'exact': the exact identity.
      poisson   'mls'  : the Laplacian of Eq. (13) is the MLS Laplacian L (Eq. vip:1);
                'vip_divgrad': the composite operator D_vip G_vip, for which the
                projected divergence equals dt times the Poisson residual.
      pressure  'incremental': r^n carries -G p^n so that phi is the pressure
                increment of Eq. (15), p^{n+1} = p^n + phi - (dt/2Re) L phi;
                'kim_moin': r^n as printed, p^{n+1} = phi - (dt/2Re) L phi;
                'incremental_interior': 'incremental' with the term
                -(dt/2Re) L phi of Eq. (15) at interior nodes only (at a boundary
                node L is a one-sided fit; the paper gives no boundary rule).
    Boundary rows: velocity Dirichlet rows hold the node's initial value; zero
    normal derivatives are imposed through the two MLS points on the inward normal
    (Operators.Nb); pressure-increment Dirichlet rows (outlet) set phi = 0.
    Problems without such a row (periodic box, closed cavities) use the bordered
    system described at the construction of P.  AB2 starts with N^{-1} = N^0.
    """

    def __init__(self, ops: Operators, Re=None, dt=None, rtol=1e-8, maxit=200000,
                 identity="exact", poisson="mls", pressure="incremental"):
        ns = ops.ns
        self.ops = ops
        self.Re = float(ns.Re if Re is None else Re)
        self.dt = float(ns.dt if dt is None else dt)
        self.rtol = rtol
        self.maxit = maxit
        self.identity = identity
        self.poisson = poisson
        if pressure not in ("incremental", "kim_moin", "incremental_interior"):
            raise ValueError(f"unknown pressure reading {pressure!r}")
        self.pressure = pressure
        N = ops.N
        k = ns.kind
        self.alpha = self.dt / (2.0 * self.Re)
        I0 = ops.D[(0, 0)] if identity == "mls" else sp.identity(N, format="csr")
        Id = sp.identity(N, format="csr")
        S = lambda m: sp.diags(m.astype(np.float64))  # noqa: E731  row selection
        Dn = ops.Nb
        inner = k == KIND_INTERIOR
        self.inner = inner
        self.u_dir = k == KIND_WALL
        self.v_dir = (k == KIND_WALL) | (k == KIND_SLIP)
        u_neu = (k == KIND_SLIP) | (k == KIND_OUTLET)
        v_neu = k == KIND_OUTLET
        self.I0 = I0
        self.Hu = (S(inner) @ (I0 - self.alpha * ops.L) + S(self.u_dir) @ Id
                   + S(u_neu) @ Dn).tocsr()
        self.Hv = (S(inner) @ (I0 - self.alpha * ops.L) + S(self.v_dir) @ Id
                   + S(v_neu) @ Dn).tocsr()
        self.Rm = (I0 + self.alpha * ops.L).tocsr()
        phi_dir = k == KIND_OUTLET
        phi_neu = (k == KIND_WALL) | (k == KIND_SLIP)
        pin_scale = -4.0 / ns.h ** 2
        if poisson == "mls":
            Lp = ops.L
        else:
            if ns.Lx > 0 or ns.Ly > 0:
                # on a periodic lattice D_vip G_vip also annihilates the checkerboard
                # modes, so the bordered system stays singular
                raise ValueError("the composite Poisson operator needs a bounded domain")
            Lp = (ops.Gx @ S(inner) @ ops.Gx + ops.Gy @ S(inner) @ ops.Gy).tocsr()
        # Boundary rows of the Poisson system are scaled by -4/h^2 so that their
        # diagonal has the sign and size of the Laplacian rows (each equation is = 0).
        P = (S(inner) @ Lp + sp.diags(phi_neu * pin_scale) @ Dn
             + sp.diags(phi_dir * pin_scale)).tocsr()
        self.bordered = not phi_dir.any()
        self.pin = -1
        if self.bordered:
            # No Dirichlet row: P is singular and, being non-symmetric, its range does
            # not contain every right-hand side.  Border it with one unknown mu that
            # removes the part of b outside the range, spread evenly over the interior
            # rows (z = indicator of the interior rows), and fix the free constant by
            # phi_k = 0 at the first interior node k:
            #     rows i != k : (P phi)_i + z_i mu = b_i
            #     row k       : (-4/h_k^2) phi_k  = 0
            #     row N       : (P phi)_k + mu     = b_k
            # (node k's own equation moves to the extra row so that no diagonal entry
            # is zero; BiCGSTAB stagnates on a zero diagonal of the bordered form).
            k0 = int(np.nonzero(inner)[0][0])
            self.pin = k0
            z = inner.astype(np.float64)
            Pb = sp.bmat([[P, sp.csr_matrix(z[:, None])],
                          [sp.csr_matrix((1, N)), None]]).tolil()
            rowk = Pb[k0].copy()
            Pb[k0] = 0.0
            Pb[k0, k0] = pin_scale[k0]
            Pb[N] = rowk
            P = Pb.tocsr()
        self.P = P
        self.b_rows = inner
        self.u = ns.u0.copy()
        self.v = ns.v0.copy()
        self.p = ns.p0.copy()
        self.phi = np.zeros(N)
        self.mu = 0.0
        self.u_bc = ns.u0.copy()
        self.v_bc = ns.v0.copy()
        self.N_prev = None
        self.nstep = 0
        self.stats = []

    def set_state(self, u, v, p, phi=None):
        self.u, self.v, self.p = (np.array(a, np.float64) for a in (u, v, p))
        self.phi = np.zeros(self.ops.N) if phi is None else np.array(phi, np.float64)
        self.mu = 0.0

    def step(self):
        ops = self.ops
        dt, al = self.dt, self.alpha
        u, v, p = self.u, self.v, self.p
        inner = self.inner
        # convection at t_n and its Adams-Bashforth extrapolation (Sec. 4)
        Nu, Nv = convection(ops, u, v)
        if self.N_prev is None:
            self.N_prev = (Nu, Nv)
        Nu_ab = 1.5 * Nu - 0.5 * self.N_prev[0]
        Nv_ab = 1.5 * Nv - 0.5 * self.N_prev[1]
        self.N_prev = (Nu, Nv)
        # Eq. (12) times dt: (I - al L) u* = (I + al L) u^n - dt [N^{n+1/2} + G p^n]
        incremental = self.pressure != "kim_moin"
        gpx = ops.Gx @ p if incremental else 0.0
        gpy = ops.Gy @ p if incremental else 0.0
        ru = np.where(inner, self.Rm @ u - dt * (Nu_ab + gpx), 0.0)
        rv = np.where(inner, self.Rm @ v - dt * (Nv_ab + gpy), 0.0)
        ru = np.where(self.u_dir, self.u_bc, ru)
        rv = np.where(self.v_dir, self.v_bc, rv)
        us, itu, resu = bicgstab(self.Hu, ru, u, self.rtol, self.maxit)
        vs, itv, resv = bicgstab(self.Hv, rv, v, self.rtol, self.maxit)
        self.ustar, self.vstar = us, vs
        # Eq. (13): L phi = div_vip(u*) / dt
        b = np.where(self.b_rows, (ops.Gx @ us + ops.Gy @ vs) / dt, 0.0)
        self.b_last = b
        if self.bordered:
            b = np.append(b, b[self.pin])
            b[self.pin] = 0.0
            x0 = np.append(self.phi, self.mu)
        else:
            x0 = self.phi
        sol, itp, resp = bicgstab(self.P, b, x0, self.rtol, self.maxit)
        phi = sol[:self.ops.N]
        self.mu = float(sol[-1]) if self.bordered else 0.0
        # Eq. (14): u^{n+1} = u* - dt grad_vip(phi) at interior nodes
        self.u = np.where(inner, us - dt * (ops.Gx @ phi), us)
        self.v = np.where(inner, vs - dt * (ops.Gy @ phi), vs)
        # Eq. (15)
        self.p = self.pressure_update(p, phi)
        self.phi = phi
        self.nstep += 1
        st = {"it_u": itu, "it_v": itv, "it_p": itp, "res_u": resu, "res_v": resv,
              "res_p": resp, "b_norm": float(np.linalg.norm(b)),
              "poisson_residual": b - self.P @ sol}
        self.stats.append({k: v for k, v in st.items() if k != "poisson_residual"})
        self.last = st
        return st

    def pressure_update(self, p, phi):
        """Eq. (15) under the pressure reading: p^{n+1} from p^n and phi^{n+1}."""
        base = p if self.pressure != "kim_moin" else 0.0
        rot = self.ops.L @ phi
        if self.pressure == "incremental_interior":
            rot = np.where(self.inner, rot, 0.0)
        return base + phi - self.alpha * rot

    def divergence(self, u=None, v=None):
        """div_vip of a velocity field at interior nodes (Sec. 4.1, item 2)."""
        u = self.u if u is None else u
        v = self.v if v is None else v
        return np.where(self.inner, self.ops.Gx @ u + self.ops.Gy @ v, 0.0)
