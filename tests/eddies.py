"""Moffatt eddies from the velocity across the symmetry axis of a triangular cavity
(Sec. 5, triangular cavity flow; Tables 1 and 2), for the host post-processing of
a GPU run.

Along the axis, eddy centres are where the velocity across the axis vanishes
(an extremum of the stream function), and an eddy's intensity is the largest
magnitude of that velocity between consecutive centres, which is where the
dividing streamline between two eddies crosses the axis.  Tables 1 and 2 report
the ratios r_n / r_(n+1) of the centres' distances from the apex and I_n / I_(n+1)
of the intensities, counted from the largest eddy.
"""
import numpy as np


def axis_eddies(r, u, r_min=0.0):
    """r: ascending distances from the apex of the axis samples; u: the velocity
    across the axis there.  Returns (centres, intensities), both ordered from the
    apex outwards, for samples with r > r_min.

    centres: zeros of u, by linear interpolation between samples of opposite sign;
    intensities: |u| at each extremum between consecutive centres, refined by the
    parabola through the largest sample and its two neighbours."""
    r = np.asarray(r, np.float64)
    u = np.asarray(u, np.float64)
    keep = r > r_min
    r, u = r[keep], u[keep]
    s = np.nonzero(np.sign(u[:-1]) * np.sign(u[1:]) < 0)[0]
    centres = r[s] - u[s] * (r[s + 1] - r[s]) / (u[s + 1] - u[s])
    intensities = []
    for a, b in zip(s[:-1], s[1:]):
        seg = np.arange(a + 1, b + 1)
        k = seg[np.argmax(np.abs(u[seg]))]
        if 0 < k < u.size - 1:
            y0, y1, y2 = np.abs(u[k - 1]), np.abs(u[k]), np.abs(u[k + 1])
            den = y0 - 2 * y1 + y2
            intensities.append(y1 - 0.125 * (y2 - y0) ** 2 / den if den != 0 else y1)
        else:
            intensities.append(np.abs(u[k]))
    return centres, np.asarray(intensities)


def moffatt_ratios(r, u, r_min=0.0):
    """(r_n / r_(n+1), I_n / I_(n+1)) counted from the outermost eddy inwards."""
    centres, inten = axis_eddies(r, u, r_min)
    c = centres[::-1]
    i = inten[::-1]
    return c[:-1] / c[1:], i[:-1] / i[1:]
