"""Force on the body of a channel_body node set, from the state of a context:

  F = sum over the body's surface nodes of t ds,
  t = -p n + (1/Re) (grad u + grad u^T) n,  n the unit normal out of the body,

which on a no-slip wall equals the traction -p n + nu du/dn of the paper's
cylinder section.  Velocity gradients come from the context's MLS derivative
tables (D10, D01), p from the state, ds = perimeter / (number of surface nodes).
Coefficients: C = 2 F / (rho U^2 D) with U = D = 1.
"""
import numpy as np
import scipy.sparse as sp

from oracle import vip_oracle as vo


class ForceProbe:
    def __init__(self, ctx, ns):
        self.ctx, self.ns = ctx, ns
        # nodes are ordered by lattice row: the body's surface nodes are the wall
        # nodes near the origin (the channel's own walls are far away)
        r = np.hypot(ns.x, ns.y)
        s = np.nonzero((ns.kind == vo.KIND_WALL) & (r < 2.0))[0]
        assert s.size == ns.meta["surface_nodes"]
        s = s[np.argsort(np.arctan2(ns.y[s], ns.x[s]))]
        xs, ys = np.append(ns.x[s], ns.x[s][0]), np.append(ns.y[s], ns.y[s][0])
        self.ds = np.sum(np.hypot(np.diff(xs), np.diff(ys))) / s.size
        self.s = s
        self.nbx, self.nby = -ns.nx[s], -ns.ny[s]  # the node set's normals point into the body

        def rows(which):
            ptr, col, val = ctx.vip_get_stencil(which)
            return sp.csr_matrix((val, col, ptr), shape=(ns.n, ns.n))[s]

        self.D10, self.D01 = rows("D10"), rows("D01")

    def coefficients(self):
        """(C_D, C_L) of the current state."""
        u, v, p, _ = self.ctx.vip_get_state()
        s, nbx, nby, Re = self.s, self.nbx, self.nby, self.ns.Re
        ux, uy, vx, vy = self.D10 @ u, self.D01 @ u, self.D10 @ v, self.D01 @ v
        tx = -p[s] * nbx + (2 * ux * nbx + (uy + vx) * nby) / Re
        ty = -p[s] * nby + ((uy + vx) * nbx + 2 * vy * nby) / Re
        return 2 * np.sum(tx) * self.ds, 2 * np.sum(ty) * self.ds


def strouhal(t, cl):
    """Dominant frequency of a uniformly sampled signal: Hann-windowed spectrum, the
    peak refined by a parabola through the log power of its three bins."""
    x = (cl - cl.mean()) * np.hanning(cl.size)
    P = np.abs(np.fft.rfft(x)) ** 2
    i = int(np.argmax(P[1:])) + 1
    a, b, c = np.log(P[i - 1]), np.log(P[i]), np.log(P[i + 1])
    return (i + 0.5 * (a - c) / (a - 2 * b + c)) / (cl.size * (t[1] - t[0]))
