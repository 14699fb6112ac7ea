"""Stepwise adaptive node distributions (workloads.channel_body(refine=...)), the
nested uniform regions of the paper's cylinder flows (Sec. 5.4, and Sec. 5.5 for
the bumpy bodies), checked on the CPU with the oracle.

  * structure: every node of level k lies on the lattice of spacing h 2^k, inside box
    k and outside box k-1; a box's edge carries only the coarser lattice's points, at
    the coarser spacing; no two nodes coincide; without `refine` the node set is the
    uniform one;
  * the MLS weights reproduce quadratics at every node, VIP and normal point of the
    adaptive set (the transitions included), as on uniform sets (1e-12);
  * a channel with one refinement box (h = 1/8 inside, 1/4 outside, Re = 20, so the
    coarse region's cell Reynolds number is 5) settles: bounded, and the change of
    its velocity over steps 800-1200 (t 25-37.5) is below 1e-2 and below half the
    change over steps 400-800 (measured 2.5e-2, then 6.2e-3, then 2.3e-3 ... 3e-4 by
    t = 75).  With the finer points on the box's edge at their own spacing the same
    channel diverges by t = 25, and at the coarser spacing it drifts without decay.
"""
import numpy as np
import pytest

import workloads as w
from oracle import vip_oracle as vo

BOX = [(-1.5, 3.0, -1.5, 1.5)]


def small(Re=20.0, refine=BOX):
    return w.channel_body(1 / 8, ("circle", 0.5), Re=Re, xlim=(-4, 8), ylim=(-3, 3), refine=refine)


def test_structure_of_the_stepwise_distribution():
    h = 1 / 16
    boxes = [(-1.0, 1.5, -1.0, 1.0), (-2.0, 3.0, -1.5, 1.5)]
    ns = w.channel_body(h, ("circle", 0.5), Re=40.0, xlim=(-4, 8), ylim=(-3, 3), refine=boxes)
    lat = np.abs(np.hypot(ns.x, ns.y) - 0.5) > 1e-9   # not a surface node of the circle
    assert (~lat).sum() == ns.meta["surface_nodes"]
    x, y, hl = ns.x[lat], ns.y[lat], ns.h[lat]
    ix, iy = (x + 4) / h, (y + 3) / h
    assert np.allclose(ix, np.round(ix)) and np.allclose(iy, np.round(iy))
    ix, iy = np.round(ix).astype(int), np.round(iy).astype(int)
    pts = set(zip(ix.tolist(), iy.tolist()))
    assert len(pts) == ix.size  # no duplicates

    def inside(k):
        x0, x1, y0, y1 = boxes[k]
        return (x >= x0 - 1e-12) & (x <= x1 + 1e-12) & (y >= y0 - 1e-12) & (y <= y1 + 1e-12)

    level = np.where(inside(0), 0, np.where(inside(1), 1, 2))
    for k in range(3):
        st = 2 ** k
        sel = level == k
        assert np.all(ix[sel] % st == 0) and np.all(iy[sel] % st == 0), k
    # a box's edge: only the coarser lattice's points, at the coarser spacing
    for k, (x0, x1, y0, y1) in enumerate(boxes):
        edge = (level == k) & (np.isclose(x, x0) | np.isclose(x, x1) | np.isclose(y, y0) | np.isclose(y, y1))
        st = 2 ** (k + 1)
        assert edge.any() and np.all(ix[edge] % st == 0) and np.all(iy[edge] % st == 0), k
        assert np.allclose(hl[edge], h * st), k
        rest = (level == k) & ~edge
        assert np.allclose(hl[rest], h * 2 ** k), k
    assert np.allclose(hl[level == 2], 4 * h)
    assert ns.meta["level_nodes"] == [int((level == k).sum()) for k in range(3)]
    # every lattice point of a box at its own spacing is a node (outside the body)
    x0, x1, y0, y1 = boxes[1]
    a, b = int(round((x0 + 4) / h)), int(round((x1 + 4) / h))
    c, d = int(round((y0 + 3) / h)), int(round((y1 + 3) / h))
    assert (a, c) in pts and (b, d) in pts and (a + 4, c) in pts and (a + 2, c) not in pts
    assert (a + 2, c + 2) in pts and (a + 1, c + 2) not in pts
    # no refinement: the uniform node set
    u1 = w.channel_body(1 / 8, ("circle", 0.5), Re=100.0, xlim=(-3, 5), ylim=(-2, 2))
    assert np.allclose(u1.h, 1 / 8) and u1.n == 2101


def test_box_edges_must_lie_on_the_outer_lattice():
    with pytest.raises(ValueError):
        w.channel_body(1 / 8, ("circle", 0.5), xlim=(-4, 8), ylim=(-3, 3), refine=[(-1.375, 3.0, -1.5, 1.5)])


def test_mls_reproduces_quadratics_across_the_transitions():
    ns = small()
    ops = vo.Operators(ns)
    x, y = ns.x, ns.y
    for (a, b), A in ops.D.items():
        for q, der in ((np.ones_like(x), {}), (x, {(1, 0): 1.0}), (y, {(0, 1): 1.0}),
                       (x * x, {(1, 0): 2 * x, (2, 0): 2.0}), (x * y, {(1, 0): y, (0, 1): x, (1, 1): 1.0}),
                       (y * y, {(0, 1): 2 * y, (0, 2): 2.0})):
            exact = q if (a, b) == (0, 0) else der.get((a, b), 0.0) * np.ones_like(x)
            scale = np.abs(A).sum(axis=1).A1 * np.max(np.abs(q)) + 1.0
            assert np.max(np.abs(A @ q - exact) / scale) <= 1e-12, ((a, b),)
    for k, I in ops.I.items():  # VIP interpolation at interior nodes
        ii = ops.interior
        qx, qy = ops.vip[k]
        for q, f in ((x * x, lambda X, Y: X * X), (x * y, lambda X, Y: X * Y)):
            v = (I @ q)[ii]
            assert np.max(np.abs(v - f(qx, qy))) <= 1e-12 * (np.max(np.abs(q)) + 1.0), k


def test_one_box_channel_settles():
    ns = small()
    fs = vo.FractionalStep(vo.Operators(ns), rtol=1e-8)
    snaps = []
    for k in range(1200):
        fs.step()
        if k + 1 in (400, 800, 1200):
            snaps.append(fs.u.copy())
    assert np.all(np.isfinite(fs.u)) and np.abs(fs.u).max() < 2.0
    d1 = np.max(np.abs(snaps[1] - snaps[0]))
    d2 = np.max(np.abs(snaps[2] - snaps[1]))
    assert d2 < 1e-2 and d2 < 0.5 * d1, (d1, d2)
