"""The seeded 3D node sets (workloads/geometry3d.py): counts, kinds, normals, jitter
bounds and periodic ranges, on the CPU."""
import numpy as np
import pytest

import workloads as w


def test_walled_box():
    ns = w.box3d(6)
    assert ns.n == 7 ** 3 and (ns.Lx, ns.Ly, ns.Lz) == (0.0, 0.0, 0.0)
    wall = ns.kind == w.KIND_WALL
    assert wall.sum() == 7 ** 3 - 5 ** 3 and np.all(ns.kind[~wall] == w.KIND_INTERIOR)
    nrm = np.stack([ns.nx, ns.ny, ns.nz], 1)
    assert np.allclose(np.linalg.norm(nrm[wall], axis=1), 1.0) and np.all(nrm[~wall] == 0.0)
    # outward: a normal step leaves the unit cube, an inward one stays inside
    out = np.stack([ns.x, ns.y, ns.z], 1)[wall] + 0.1 * nrm[wall]
    inn = np.stack([ns.x, ns.y, ns.z], 1)[wall] - 0.1 * nrm[wall]
    assert np.all(np.any((out < 0) | (out > 1), axis=1)) and np.all((inn > 0) & (inn < 1))


def test_jitter_and_periodic_ranges():
    a, b = w.box3d(8, jitter=0.3, seed=4), w.box3d(8, jitter=0.3, seed=4)
    assert np.array_equal(a.x, b.x)                       # seeded
    plain = w.box3d(8)
    d = np.abs(np.stack([a.x - plain.x, a.y - plain.y, a.z - plain.z], 1))
    inner = a.kind == w.KIND_INTERIOR
    assert d[inner].max() <= 0.3 * a.h[0] + 1e-15 and np.all(d[~inner] == 0.0)
    p = w.box3d(7, periodic=True, jitter=0.3, seed=6, length=2.0)
    assert p.n == 7 ** 3 and np.all(p.kind == w.KIND_INTERIOR) and (p.Lx, p.Ly, p.Lz) == (2.0, 2.0, 2.0)
    for c in (p.x, p.y, p.z):
        assert np.all((c >= 0.0) & (c < 2.0))
    with pytest.raises(ValueError):
        w.box3d(4, jitter=0.5)


def test_sphere_in_box():
    h, R = 1 / 8, 0.3
    ns = w.sphere_in_box3d(h, radius=R)
    pts = np.stack([ns.x, ns.y, ns.z], 1)
    r = np.linalg.norm(pts, axis=1)
    surf = np.isclose(r, R)
    assert surf.sum() == ns.meta["surface_nodes"] == round(4 * np.pi * R * R / (h * h))
    assert np.all(ns.kind[surf] == w.KIND_WALL)
    nrm = np.stack([ns.nx, ns.ny, ns.nz], 1)
    assert np.allclose(nrm[surf], -pts[surf] / R)          # out of the fluid: into the sphere
    lattice = ~surf
    assert np.all(r[lattice] > R + 0.55 * h - 1e-12)      # the clearance around the sphere
    with pytest.raises(ValueError):
        w.sphere_in_box3d(0.4)                            # the box [-0.75, 0.75] is 3.75 spacings
