"""Pins of the oracle's cell metric (Sect. 2.2) on the cylindrical mesh by plane
geometry in Cartesian coordinates, independent of its closed forms.

A cell of the logarithmic mesh (Sect. 2.3) is the annular sector
r- <= r <= r+, theta- <= theta <= theta+, extruded over dz.  Its outline in
the (x, y) plane, sampled finely along both arcs, is a polygon: the shoelace
formula gives the sector's area (the z-face area; times dz, the volume), the
lengths of the two arcs as polylines give the radial faces (times dz), and
the straight edge gives the theta faces (times dz).  The polygon converges to
the sector as the sampling refines, so the bar is the sampling error.
"""
import numpy as np
import pytest

import oracle
import synthetic as syn


def _sector(rm, rp, t0, t1, n=20000):
    th = np.linspace(t0, t1, n)
    outer = np.stack([rp * np.cos(th), rp * np.sin(th)], 1)
    inner = np.stack([rm * np.cos(th[::-1]), rm * np.sin(th[::-1])], 1)
    poly = np.concatenate([outer, inner])
    x, y = poly[:, 0], poly[:, 1]
    area = 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))
    arc = lambda p: np.sqrt((np.diff(p, axis=0) ** 2).sum(1)).sum()
    edge = np.hypot(*(outer[0] - inner[-1]))
    return area, arc(inner), arc(outer), edge


@pytest.mark.parametrize("w", [syn.scaled(syn.VORTEX, 10, 12, 6), syn.scaled(syn.EXPLOSION, 16, 8, 1)],
                         ids=["disc", "explosion"])
def test_cell_metric_is_the_annular_sector(w):
    o = oracle.Oracle(w)
    _, rf = o.coords(0)
    dth = (w.x1[1] - w.x0[1]) / w.nth
    dz = (w.x1[2] - w.x0[2]) / w.nz
    for i in (0, w.nr // 2, w.nr - 1):
        V, a_lo_r, a_lo_t, a_lo_z, a_hi_r, a_hi_t, a_hi_z, maxA = o.metric(i)
        area, arc_in, arc_out, edge = _sector(rf[i], rf[i + 1], 0.3, 0.3 + dth)
        tol = 1e-7
        assert V == pytest.approx(area * dz, rel=tol)
        assert a_lo_z == pytest.approx(area, rel=tol) and a_hi_z == a_lo_z
        assert a_lo_r == pytest.approx(arc_in * dz, rel=tol)
        assert a_hi_r == pytest.approx(arc_out * dz, rel=tol)
        assert a_lo_t == pytest.approx(edge * dz, rel=1e-12) and a_hi_t == a_lo_t
        assert maxA == max(a_hi_r, a_hi_t, a_hi_z)
