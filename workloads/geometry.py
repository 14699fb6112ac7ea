"""Node sets and initial states for the VIP solver workloads (Sec. 5 of the paper).

Node-kind encoding (the input format of the node set, one byte per node):

  KIND_INTERIOR  momentum and Poisson equations are collocated at the node.
  KIND_WALL      velocity Dirichlet (value = the initial state at the node, held
                 fixed), pressure-increment Neumann (normal derivative zero).
                 Used for no-slip walls, the moving lid and the inflow boundary.
  KIND_SLIP      tangential velocity Neumann, normal velocity Dirichlet, pressure
                 increment Neumann (the top/bottom channel walls, "v = 0, t_x = 0",
                 Sec. 5.4).
  KIND_OUTLET    velocity Neumann, pressure increment Dirichlet zero (traction
                 free outflow, Sec. 5.4).

Normals (nx, ny) are unit outward normals of the fluid domain at boundary nodes
and zero at interior nodes.  h is the local node spacing.

Geometric conventions that keep every virtual interpolation point inside the
closed fluid domain: nodes lie on the straight walls of the box domains, and
lattice nodes closer than CLEARANCE*h to a curved or slanted wall are removed, so
a point half a spacing away along a coordinate axis never crosses a wall.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy.spatial import cKDTree

KIND_INTERIOR = 0
KIND_WALL = 1
KIND_SLIP = 2
KIND_OUTLET = 3

# Lattice nodes nearer than CLEARANCE*h to a curved/slanted wall are dropped.
CLEARANCE = 0.55
# Local spacing factor near the 60-degree corners of the triangular cavities.
CORNER_SUPPORT = 1.6


@dataclass
class NodeSet:
    name: str
    x: np.ndarray
    y: np.ndarray
    kind: np.ndarray
    nx: np.ndarray
    ny: np.ndarray
    h: np.ndarray
    Lx: float
    Ly: float
    u0: np.ndarray
    v0: np.ndarray
    p0: np.ndarray
    Re: float
    dt: float
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def counts(self) -> dict:
        return {k: int(np.sum(self.kind == v)) for k, v in
                (("interior", KIND_INTERIOR), ("wall", KIND_WALL),
                 ("slip", KIND_SLIP), ("outlet", KIND_OUTLET))}


def taylor_green(x, y, t, Re):
    """Closed-form decaying vortices (Sec. 5.1) in the form that satisfies Eqs. (1)-(2).

    u = -cos x sin y e^{-2t/Re}, v = sin x cos y e^{-2t/Re},
    p = -(cos 2x + cos 2y) e^{-4t/Re} / 4.
    """
    e = np.exp(-2.0 * t / Re)
    u = -np.cos(x) * np.sin(y) * e
    v = np.sin(x) * np.cos(y) * e
    p = -0.25 * (np.cos(2.0 * x) + np.cos(2.0 * y)) * e * e
    return u, v, p


def _finish(name, x, y, kind, nx, ny, h, Lx, Ly, u0, v0, p0, Re, dt, ymin, meta=None):
    """Order nodes by lattice row, then by x (keeps stencil neighbours close in memory)."""
    hh = float(np.min(h))
    row = np.floor((y - ymin) / hh + 0.5).astype(np.int64)
    order = np.lexsort((x, row))
    f = lambda a: np.ascontiguousarray(a[order])  # noqa: E731
    return NodeSet(name, f(x).astype(np.float64), f(y).astype(np.float64),
                   f(kind).astype(np.uint8), f(nx).astype(np.float64),
                   f(ny).astype(np.float64), f(h).astype(np.float64),
                   float(Lx), float(Ly), f(u0).astype(np.float64),
                   f(v0).astype(np.float64), f(p0).astype(np.float64),
                   float(Re), float(dt), meta or {})


def periodic_box(n: int, Re: float = 100.0, dt: float = 1e-3, t0: float = 0.0) -> NodeSet:
    """Decaying vortices on the periodic box [0, 2pi)^2 with n x n regular nodes."""
    L = 2.0 * np.pi
    h = L / n
    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    x = (i * h).ravel().astype(np.float64)
    y = (j * h).ravel().astype(np.float64)
    N = x.size
    u0, v0, p0 = taylor_green(x, y, t0, Re)
    z = np.zeros(N)
    return _finish(f"periodic{n}", x, y, np.zeros(N, np.uint8), z, z.copy(),
                   np.full(N, h), L, L, u0, v0, p0, Re, dt, 0.0,
                   {"h": h, "n": n, "t0": t0})


def cavity(n: int, Re: float = 1000.0, dt: float | None = None, lid: float = 1.0) -> NodeSet:
    """Lid-driven square cavity [0,1]^2, n x n regular nodes with nodes on the walls.

    The lid (top wall) moves with u = lid; its two end nodes take the wall value 0.
    """
    h = 1.0 / (n - 1)
    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    i = i.ravel()
    j = j.ravel()
    x = i * h
    y = j * h
    N = x.size
    kind = np.zeros(N, np.uint8)
    nx = np.zeros(N)
    ny = np.zeros(N)
    nx[i == 0] -= 1.0
    nx[i == n - 1] += 1.0
    ny[j == 0] -= 1.0
    ny[j == n - 1] += 1.0
    bnd = (i == 0) | (i == n - 1) | (j == 0) | (j == n - 1)
    kind[bnd] = KIND_WALL
    nrm = np.hypot(nx, ny)
    nx[bnd] /= nrm[bnd]
    ny[bnd] /= nrm[bnd]
    u0 = np.zeros(N)
    u0[(j == n - 1) & (i > 0) & (i < n - 1)] = lid
    if dt is None:
        dt = 0.25 * h
    return _finish(f"cavity{n}", x, y, kind, nx, ny, np.full(N, h), 0.0, 0.0,
                   u0, np.zeros(N), np.zeros(N), Re, dt, 0.0, {"h": h, "n": n})


def _radial_body(spec):
    """Return r(theta), r'(theta) for a star-shaped body given by its spec."""
    kind = spec[0]
    if kind == "circle":
        R = float(spec[1])
        return (lambda t: np.full_like(t, R)), (lambda t: np.zeros_like(t)), R
    if kind == "sines":  # r = r0 + sum a_k sin(k theta)
        r0 = float(spec[1])
        terms = [(float(a), float(k)) for a, k in spec[2]]
        r = lambda t: r0 + sum(a * np.sin(k * t) for a, k in terms)  # noqa: E731
        dr = lambda t: sum(a * k * np.cos(k * t) for a, k in terms)  # noqa: E731
        return r, dr, r0 + sum(abs(a) for a, _ in terms)
    if kind == "bumps":  # r = r0 (1 + gamma cos(m theta)), the family of Sec. 5.5
        r0, gamma, m = float(spec[1]), float(spec[2]), float(spec[3])
        return ((lambda t: r0 * (1 + gamma * np.cos(m * t))),
                (lambda t: -r0 * gamma * m * np.sin(m * t)), r0 * (1 + gamma))
    raise ValueError(f"unknown body {spec!r}")


def _stepwise_lattice(h, xlim, ylim, refine):
    """Lattice nodes of a stepwise adaptive distribution: spacing h inside the first
    box of `refine` (x0, x1, y0, y1), 2h between the first and the second, ..., and
    h 2^K outside the last of the K boxes, all lattices sharing the origin
    (xlim[0], ylim[0]).  A node of level k lies in box k (the channel for k = K) and
    not in box k-1 (closed), whose edge nodes belong to the finer level.  Returns the
    finest-lattice indices (ii, jj) of the nodes, their level and the lattice size."""
    K = len(refine)
    nxl = int(round((xlim[1] - xlim[0]) / h)) + 1
    nyl = int(round((ylim[1] - ylim[0]) / h)) + 1
    boxes = []
    for k, (x0, x1, y0, y1) in enumerate(refine):
        step = 2 ** (k + 1)   # the box edges lie on the lattice outside them
        e = [(x0 - xlim[0]) / h, (x1 - xlim[0]) / h, (y0 - ylim[0]) / h, (y1 - ylim[0]) / h]
        ei = [int(round(v)) for v in e]
        if any(abs(a - b) > 1e-9 for a, b in zip(e, ei)) or any(v % step for v in ei):
            raise ValueError(f"box {k} edges must lie on the lattice of spacing {step} h")
        boxes.append(ei)
    iis, jjs, levs = [], [], []
    for k in range(K + 1):
        st = 2 ** k
        jj, ii = np.meshgrid(np.arange(0, nyl, st), np.arange(0, nxl, st), indexing="ij")
        ii, jj = ii.ravel(), jj.ravel()
        keep = np.ones(ii.size, bool)
        if k < K:
            a0, a1, b0, b1 = boxes[k]
            keep &= (ii >= a0) & (ii <= a1) & (jj >= b0) & (jj <= b1)
            # the box's edge carries only the coarser lattice's points
            edge = (ii == a0) | (ii == a1) | (jj == b0) | (jj == b1)
            keep &= ~(edge & ((ii % (2 * st) != 0) | (jj % (2 * st) != 0)))
        if k > 0:
            a0, a1, b0, b1 = boxes[k - 1]
            keep &= ~((ii >= a0) & (ii <= a1) & (jj >= b0) & (jj <= b1))
        iis.append(ii[keep])
        jjs.append(jj[keep])
        levs.append(np.full(int(keep.sum()), k, np.int64))
    return np.concatenate(iis), np.concatenate(jjs), np.concatenate(levs), nxl, nyl


def channel_body(h: float, body=("circle", 0.5), Re: float = 100.0, dt: float | None = None,
                 xlim=(-8.0, 24.0), ylim=(-8.0, 8.0), name: str | None = None,
                 refine=()) -> NodeSet:
    """Uniform inflow past a star-shaped body centred at the origin (Sec. 5.4-5.5).

    Background lattice of spacing h over the channel; lattice nodes inside the body
    or within CLEARANCE*h of its surface are removed; boundary nodes are placed on the
    surface at arc-length spacing close to h.  Inflow (x = xmin): u = 1, v = 0.
    Outflow (x = xmax): traction free.  Top/bottom: v = 0 with zero shear.

    refine: the stepwise adaptive distribution of the paper's cylinder flows (Sec. 5.4,
    used again in Sec. 5.5): nested boxes (x0, x1, y0, y1), innermost first, with
    spacing h in the first and doubling outward (h 2^K outside the last); each box's
    edges lie on the lattice outside it.  A node's h_local is its lattice's spacing,
    except on a box's edge, which carries only the coarser lattice's points, with the
    coarser spacing (reading: the paper gives no rule for the transition; with the
    finer points and spacing on the edge the flow develops a growing mode at the box
    corners, with the finer points at the coarser spacing a slower one).  The body
    must lie in the first box.  The central VIP fluxes also need the cell Reynolds
    number Re h 2^K of the coarsest region to stay moderate, as on a uniform lattice.
    """
    rfun, drfun, rmax = _radial_body(body)
    ii, jj, lev, nxl, nyl = _stepwise_lattice(h, xlim, ylim, tuple(refine))
    x = xlim[0] + ii * h
    y = ylim[0] + jj * h
    # body surface, densely sampled for the clearance test
    ts = np.linspace(0.0, 2 * np.pi, int(2 * np.pi * rmax / (h / 64)) + 64, endpoint=False)
    rs = rfun(ts)
    cx, cy = rs * np.cos(ts), rs * np.sin(ts)
    rad = np.hypot(x, y)
    near = rad < rmax + 2 * h
    keep = np.ones(x.size, bool)
    idx = np.nonzero(near)[0]
    th = np.arctan2(y[idx], x[idx])
    inside = rad[idx] < rfun(th)
    d, _ = cKDTree(np.stack([cx, cy], 1)).query(np.stack([x[idx], y[idx]], 1))
    keep[idx[inside | (d < CLEARANCE * h)]] = False
    x, y, ii, jj, lev = x[keep], y[keep], ii[keep], jj[keep], lev[keep]
    N0 = x.size
    kind = np.zeros(N0, np.uint8)
    nx = np.zeros(N0)
    ny = np.zeros(N0)
    inlet = ii == 0
    outlet = ii == nxl - 1
    bot = jj == 0
    top = jj == nyl - 1
    kind[bot | top] = KIND_SLIP
    kind[outlet] = KIND_OUTLET
    kind[inlet] = KIND_WALL
    nx[inlet] -= 1.0
    nx[outlet] += 1.0
    ny[bot] -= 1.0
    ny[top] += 1.0
    bnd = inlet | outlet | bot | top
    nrm = np.hypot(nx, ny)
    nx[bnd] /= nrm[bnd]
    ny[bnd] /= nrm[bnd]
    u0 = np.ones(N0)
    # surface nodes at (nearly) equal arc length
    tf = np.linspace(0.0, 2 * np.pi, 200001)
    rf = rfun(tf)
    px, py = rf * np.cos(tf), rf * np.sin(tf)
    s = np.concatenate([[0.0], np.cumsum(np.hypot(np.diff(px), np.diff(py)))])
    M = max(8, int(round(s[-1] / h)))
    tb = np.interp(np.arange(M) * s[-1] / M, s, tf)
    rb, drb = rfun(tb), drfun(tb)
    bx, by = rb * np.cos(tb), rb * np.sin(tb)
    tx = drb * np.cos(tb) - rb * np.sin(tb)
    ty = drb * np.sin(tb) + rb * np.cos(tb)
    tn = np.hypot(tx, ty)
    # outward normal of the fluid domain points into the body
    bnx, bny = -ty / tn, tx / tn
    x = np.concatenate([x, bx])
    y = np.concatenate([y, by])
    kind = np.concatenate([kind, np.full(M, KIND_WALL, np.uint8)])
    nx = np.concatenate([nx, bnx])
    ny = np.concatenate([ny, bny])
    u0 = np.concatenate([u0, np.zeros(M)])
    N = x.size
    if dt is None:
        dt = 0.25 * h
    hl = h * 2.0 ** lev
    for k, (x0, x1, y0, y1) in enumerate(refine):
        # nodes of level k on the edge of box k: the spacing outside the box
        xl, yl = x[:N0], y[:N0]
        inb = (xl >= x0 - 1e-12) & (xl <= x1 + 1e-12) & (yl >= y0 - 1e-12) & (yl <= y1 + 1e-12)
        onb = np.isclose(xl, x0) | np.isclose(xl, x1) | np.isclose(yl, y0) | np.isclose(yl, y1)
        hl[(lev == k) & inb & onb] = h * 2.0 ** (k + 1)
    hl = np.concatenate([hl, np.full(M, h)])
    meta = {"h": h, "body": body, "surface_nodes": M, "lattice": (nxl, nyl)}
    if refine:
        meta["refine"] = tuple(tuple(b) for b in refine)
        meta["level_nodes"] = [int((lev == k).sum()) for k in range(len(refine) + 1)]
    return _finish(name or f"channel_{body[0]}_h{int(round(1 / h))}", x, y, kind, nx, ny,
                   hl, 0.0, 0.0, u0, np.zeros(N), np.zeros(N), Re, dt, ylim[0], meta)


def triangle_cavity(n_edge: int, Re: float = 100.0, dt: float | None = None,
                    name: str | None = None) -> NodeSet:
    """Equilateral triangular cavity with unit edges, lid on the top edge (Sec. 5.3 family).

    Vertices (0,0), (1,0) (the lid) and (1/2, -sqrt(3)/2).  Lattice spacing
    h = 1/(n_edge-1); edge nodes at spacing h; lattice nodes within CLEARANCE*h of
    a slanted edge are removed.  Nodes within 3h of a vertex get
    h_local = CORNER_SUPPORT*h so that their support covers enough nodes for a
    quadratic fit in the narrow corners.
    """
    n = int(n_edge)
    h = 1.0 / (n - 1)
    H = np.sqrt(3.0) / 2.0
    A = np.array([0.0, 0.0])
    B = np.array([1.0, 0.0])
    C = np.array([0.5, -H])
    xs, ys, ks, nxs, nys, us = [], [], [], [], [], []
    # lid row
    i = np.arange(n)
    xs.append(i * h)
    ys.append(np.zeros(n))
    ks.append(np.full(n, KIND_WALL, np.uint8))
    lnx = np.zeros(n)
    lny = np.ones(n)
    c30, s30 = np.cos(np.pi / 6), np.sin(np.pi / 6)
    lnx[0], lny[0] = -c30, s30
    lnx[-1], lny[-1] = c30, s30
    nxs.append(lnx)
    nys.append(lny)
    ul = np.ones(n)
    ul[0] = ul[-1] = 0.0
    us.append(ul)
    # slanted edges (apex once)
    t = np.arange(1, n) / (n - 1)
    left = A[None, :] + t[:, None] * (C - A)[None, :]
    t2 = np.arange(1, n - 1) / (n - 1)
    right = B[None, :] + t2[:, None] * (C - B)[None, :]
    lnrm = np.tile([-c30, -s30], (n - 1, 1))
    lnrm[-1] = [0.0, -1.0]
    rnrm = np.tile([c30, -s30], (n - 2, 1))
    for P, Nn in ((left, lnrm), (right, rnrm)):
        xs.append(P[:, 0])
        ys.append(P[:, 1])
        ks.append(np.full(P.shape[0], KIND_WALL, np.uint8))
        nxs.append(Nn[:, 0])
        nys.append(Nn[:, 1])
        us.append(np.zeros(P.shape[0]))
    # interior lattice
    nrow = int(np.floor(H / h))
    jj, ii = np.meshgrid(np.arange(1, nrow + 1), np.arange(n), indexing="ij")
    px = (ii * h).ravel()
    py = (-jj * h).ravel()
    # signed distances to the slanted edges (positive inside)
    dl = (px - A[0]) * c30 + (py - A[1]) * s30
    dr = -(px - B[0]) * c30 + (py - B[1]) * s30
    ok = (dl >= CLEARANCE * h) & (dr >= CLEARANCE * h)
    xs.append(px[ok])
    ys.append(py[ok])
    ks.append(np.zeros(int(ok.sum()), np.uint8))
    nxs.append(np.zeros(int(ok.sum())))
    nys.append(np.zeros(int(ok.sum())))
    us.append(np.zeros(int(ok.sum())))
    x = np.concatenate(xs)
    y = np.concatenate(ys)
    N = x.size
    hl = np.full(N, h)
    for V in (A, B, C):  # narrow 60-degree corners: widen the support there
        hl[np.hypot(x - V[0], y - V[1]) < 3 * h] = CORNER_SUPPORT * h
    if dt is None:
        dt = 0.25 * h
    return _finish(name or f"triangle{n}", x, y, np.concatenate(ks), np.concatenate(nxs),
                   np.concatenate(nys), hl, 0.0, 0.0, np.concatenate(us), np.zeros(N),
                   np.zeros(N), Re, dt, -H - h, {"h": h, "n_edge": n})


def wedge_cavity(n_base: int, height: float = 2.0, Re: float = 1.0, dt: float | None = None,
                 apex_support: float = CORNER_SUPPORT, name: str | None = None) -> NodeSet:
    """Isosceles triangular cavity of the Moffatt-eddy flow (Sec. 5, triangular cavity
    flow): base 1 (the lid, on top), apex `height` below the base's midpoint.  The
    default height 2 gives the apex angle 2 atan(1/4) = 28.072 degrees.

    Vertices (0,0), (1,0) (the lid) and (1/2, -height).  Lattice spacing
    h = 1/(n_base-1) over the bounding box; edge nodes at spacing close to h along
    each slanted edge; lattice nodes within CLEARANCE*h of a slanted edge are removed.
    Normals point out of the cavity; at a vertex they bisect the two edges' normals.
    Nodes within 3h / sin(apex half-angle) of the apex get h_local = apex_support*h;
    the lid corners (76 degrees at the default height) keep h: a wider support
    there made the flow unstable.  Lid u = 1 (its end nodes 0), all else at rest.
    """
    n = int(n_base)
    h = 1.0 / (n - 1)
    A, B, C = np.array([0.0, 0.0]), np.array([1.0, 0.0]), np.array([0.5, -float(height)])
    L = float(np.hypot(0.5, height))
    nl = np.array([-height, -0.5]) / L      # outward normal of the left edge A-C
    nr = np.array([height, -0.5]) / L       # outward normal of the right edge B-C
    xs, ys, nxs, nys, us = [], [], [], [], []
    # lid row, corners included
    i = np.arange(n)
    xs.append(i * h)
    ys.append(np.zeros(n))
    lid_n = np.tile([0.0, 1.0], (n, 1))
    for k, side in ((0, nl), (n - 1, nr)):
        v = lid_n[k] + side
        lid_n[k] = v / np.hypot(*v)
    nxs.append(lid_n[:, 0])
    nys.append(lid_n[:, 1])
    ul = np.ones(n)
    ul[0] = ul[-1] = 0.0
    us.append(ul)
    # slanted edges without the lid corners; the apex once, on the left edge
    m = max(2, int(round(L / h)))
    t = np.arange(1, m + 1) / m
    left = A[None, :] + t[:, None] * (C - A)[None, :]
    right = B[None, :] + t[:-1, None] * (C - B)[None, :]
    lnrm = np.tile(nl, (m, 1))
    lnrm[-1] = [0.0, -1.0]
    rnrm = np.tile(nr, (m - 1, 1))
    for P, Nn in ((left, lnrm), (right, rnrm)):
        xs.append(P[:, 0])
        ys.append(P[:, 1])
        nxs.append(Nn[:, 0])
        nys.append(Nn[:, 1])
        us.append(np.zeros(P.shape[0]))
    nb = sum(a.size for a in xs)
    # interior lattice
    nrow = int(np.floor(height / h))
    jj, ii = np.meshgrid(np.arange(1, nrow + 1), np.arange(n), indexing="ij")
    px = (ii * h).ravel()
    py = (-jj * h).ravel()
    dl = -((px - A[0]) * nl[0] + (py - A[1]) * nl[1])   # distances inside the edges
    dr = -((px - B[0]) * nr[0] + (py - B[1]) * nr[1])
    ok = (dl >= CLEARANCE * h) & (dr >= CLEARANCE * h)
    xs.append(px[ok])
    ys.append(py[ok])
    nxs.append(np.zeros(int(ok.sum())))
    nys.append(np.zeros(int(ok.sum())))
    us.append(np.zeros(int(ok.sum())))
    x, y = np.concatenate(xs), np.concatenate(ys)
    N = x.size
    kind = np.zeros(N, np.uint8)
    kind[:nb] = KIND_WALL
    hl = np.full(N, h)
    half = np.arctan2(0.5, height)
    hl[np.hypot(x - C[0], y - C[1]) < 3 * h / np.sin(half)] = apex_support * h
    if dt is None:
        dt = 0.25 * h
    return _finish(name or f"wedge{n}", x, y, kind, np.concatenate(nxs), np.concatenate(nys), hl,
                   0.0, 0.0, np.concatenate(us), np.zeros(N), np.zeros(N), Re, dt, -height - h,
                   {"h": h, "n_base": n, "apex_angle_deg": float(np.degrees(2 * half))})


def triangle_batch(count: int = 64, seed: int = 20140126, lo: int = 64, hi: int = 512):
    """Seeded batch of equilateral lid-driven cavities: n_edge ~ U{lo..hi}, Re ~ U[100, 1000]."""
    rng = np.random.default_rng(seed)
    n_edge = rng.integers(lo, hi + 1, size=count)
    Re = rng.uniform(100.0, 1000.0, size=count)
    return [triangle_cavity(int(n), float(r), name=f"triangle{int(n)}_Re{r:.0f}")
            for n, r in zip(n_edge, Re)]


def workload(name: str) -> NodeSet:
    """The named workloads at their full sizes."""
    if name == "taylor_green_32":
        return periodic_box(32, Re=100.0, dt=1e-3)
    if name == "cavity_256":
        return cavity(256, Re=1000.0)
    if name == "cylinder_h32":
        return channel_body(1.0 / 32, ("circle", 0.5), Re=100.0)
    if name == "bumpy_h64":
        return channel_body(1.0 / 64, ("sines", 1.0, [(0.05, 12), (0.02, 31)]), Re=200.0,
                            name="bumpy_h64")
    raise KeyError(name)
