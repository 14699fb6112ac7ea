"""Three-dimensional node sets for the 3D extension of the VIP operator build
(the paper's introduction and Sec. 3 state that the method carries over to three
dimensions with the ten-term quadratic basis; it shows no 3D flow).

The encoding is that of the 2D node sets: one kind byte per node (KIND_INTERIOR,
KIND_WALL, ...), unit outward normals of the fluid domain at boundary nodes (zero
at interior nodes) and the local node spacing h.  Periodic lengths Lx, Ly, Lz are
0 for a non-periodic direction.

Geometry only: no weight, fit or operator is computed here.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .geometry import CLEARANCE, KIND_INTERIOR, KIND_WALL


@dataclass
class NodeSet3:
    name: str
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    kind: np.ndarray
    nx: np.ndarray
    ny: np.ndarray
    nz: np.ndarray
    h: np.ndarray
    Lx: float
    Ly: float
    Lz: float
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.size)


def _finish(name, x, y, z, kind, nrm, h, L, meta):
    f = lambda a: np.ascontiguousarray(a, dtype=np.float64)  # noqa: E731
    return NodeSet3(name, f(x), f(y), f(z), np.ascontiguousarray(kind, dtype=np.uint8),
                    f(nrm[:, 0]), f(nrm[:, 1]), f(nrm[:, 2]), f(h), *map(float, L), meta)


def box3d(n: int, periodic: bool = False, jitter: float = 0.0, seed: int = 3,
          length: float = 1.0) -> NodeSet3:
    """The cube [0, length]^3 on a lattice of spacing h = length / n.

    periodic: n^3 nodes i h (i = 0 .. n-1), all interior, periods (length, length,
    length).  Otherwise (n+1)^3 nodes; nodes on the faces are KIND_WALL with the
    outward normal of their face (edges and corners: the normalised sum of their
    faces' normals).  jitter > 0 moves every interior node by a seeded uniform
    offset in [-jitter h, jitter h] per coordinate (jitter < 0.5)."""
    if not 0.0 <= jitter < 0.5:
        raise ValueError("jitter must lie in [0, 0.5)")
    h = length / n
    m = n if periodic else n + 1
    i = np.arange(m, dtype=np.float64) * h
    X, Y, Z = (a.ravel() for a in np.meshgrid(i, i, i, indexing="ij"))
    nrm = np.zeros((X.size, 3))
    if not periodic:
        for k, c in enumerate((X, Y, Z)):
            nrm[np.isclose(c, 0.0), k] -= 1.0
            nrm[np.isclose(c, length), k] += 1.0
    on_wall = np.any(nrm != 0.0, axis=1)
    nrm[on_wall] /= np.linalg.norm(nrm[on_wall], axis=1)[:, None]
    kind = np.where(on_wall, KIND_WALL, KIND_INTERIOR).astype(np.uint8)
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        d = rng.uniform(-jitter * h, jitter * h, size=(X.size, 3))
        d[on_wall] = 0.0
        X, Y, Z = X + d[:, 0], Y + d[:, 1], Z + d[:, 2]
        if periodic:
            X, Y, Z = np.mod(X, length), np.mod(Y, length), np.mod(Z, length)
    L = (length, length, length) if periodic else (0.0, 0.0, 0.0)
    return _finish(f"box3d_{n}{'_periodic' if periodic else ''}", X, Y, Z, kind, nrm,
                   np.full(X.size, h), L, {"n": n, "jitter": jitter, "seed": seed})


def _fibonacci_sphere(count: int):
    """count nearly equally spaced unit vectors (the golden-angle spiral)."""
    k = np.arange(count, dtype=np.float64) + 0.5
    zc = 1.0 - 2.0 * k / count
    r = np.sqrt(np.maximum(0.0, 1.0 - zc * zc))
    th = np.pi * (3.0 - np.sqrt(5.0)) * k
    return np.stack([r * np.cos(th), r * np.sin(th), zc], axis=1)


def sphere_in_box3d(h: float, radius: float = 0.3, half: float = 0.75) -> NodeSet3:
    """A sphere of the given radius at the centre of the box [-half, half]^3.

    Lattice nodes of spacing h (the box must hold a whole number of spacings) on
    and inside the box, minus those closer than CLEARANCE h to the sphere's
    surface or inside it; the box faces are KIND_WALL as in box3d; the sphere
    carries round(4 pi radius^2 / h^2) KIND_WALL nodes on a golden-angle spiral,
    each with the fluid's outward normal (pointing into the sphere)."""
    m = int(round(2 * half / h))
    if abs(m * h - 2 * half) > 1e-9 * half:
        raise ValueError("the box must hold a whole number of spacings")
    i = -half + np.arange(m + 1, dtype=np.float64) * h
    X, Y, Z = (a.ravel() for a in np.meshgrid(i, i, i, indexing="ij"))
    r = np.sqrt(X * X + Y * Y + Z * Z)
    keep = r > radius + CLEARANCE * h
    X, Y, Z = X[keep], Y[keep], Z[keep]
    nrm = np.zeros((X.size, 3))
    for k, c in enumerate((X, Y, Z)):
        nrm[np.isclose(c, -half), k] -= 1.0
        nrm[np.isclose(c, half), k] += 1.0
    on_wall = np.any(nrm != 0.0, axis=1)
    nrm[on_wall] /= np.linalg.norm(nrm[on_wall], axis=1)[:, None]
    kind = np.where(on_wall, KIND_WALL, KIND_INTERIOR).astype(np.uint8)
    count = int(round(4.0 * np.pi * radius * radius / (h * h)))
    e = _fibonacci_sphere(count)
    S = radius * e
    X = np.concatenate([X, S[:, 0]])
    Y = np.concatenate([Y, S[:, 1]])
    Z = np.concatenate([Z, S[:, 2]])
    kind = np.concatenate([kind, np.full(count, KIND_WALL, np.uint8)])
    nrm = np.concatenate([nrm, -e])
    return _finish(f"sphere3d_h{int(round(1 / h))}", X, Y, Z, kind, nrm, np.full(X.size, h),
                   (0.0, 0.0, 0.0), {"radius": radius, "half": half, "surface_nodes": count})
