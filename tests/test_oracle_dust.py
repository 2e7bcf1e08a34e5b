"""Analytic dust pins of the oracle (Sect. 2.9 drag in the disc of App. A).

Settling: in a hydrostatic gas column, dust falls at the terminal velocity
relative to the gas, w_d - w_g = t_s f_z (gravity balanced by drag); with a
tiny dust-to-gas ratio the gas does not move.  The semi-implicit drag
update has this as its exact fixed point, whatever the step length.

Radial drift (Nakagawa, Sekiya & Hayashi 1986, dust-to-gas ratio -> 0): in a
gas disc rotating eta v_K slower than Keplerian, dust drifts inward at
v_r = -2 St eta v_K / (1 + St^2), with eta v_K = v_K - v_gas taken from the
equilibrium of App. A at the midplane.
"""
import math
from dataclasses import replace

import numpy as np
import pytest

import oracle
import synthetic as syn


def settling_workload():
    return replace(syn.VORTEX, name="settling_column_4x4x32", nr=4, nth=4, nz=32, x0=(0.97, 0.0, -0.15),
                   x1=(1.03, 2 * math.pi / 64, 0.15), vortices=(), dust_ratio=1e-4, dust_noise=0.0, stokes=0.01,
                   omega_frame=1.0)


def drift_workload():
    return replace(syn.VORTEX, name="radial_drift_24x4x4", nr=24, nth=4, nz=4, x0=(0.7, 0.0, -0.01),
                   x1=(1.4, 2 * math.pi / 64, 0.01), vortices=(), dust_ratio=1e-4, dust_noise=0.0, stokes=0.1,
                   omega_frame=1.0)


def settling_error(w, E, zc, rc):
    """Relative error of w_d - w_g against t_s f_z at |z| < 0.1."""
    R = rc[None, None, :]
    Z = zc[:, None, None]
    fz = -w.gm * Z / (R * R + Z * Z) ** 1.5
    ts = w.stokes / np.sqrt(w.gm / R ** 3)
    dw = E[7] / E[8] - E[2] / E[4]
    sel = np.abs(zc) < 0.1
    return (np.abs(dw - ts * fz)[sel] / np.abs(ts * fz)[sel]).max()


def drift_error(w, E, rc, eq_vtheta):
    """Relative error of the dust radial velocity against NSH at 0.85 < r < 1.2,
    away from the vertical boundaries (the outermost z cells exchange dust
    with empty ghosts)."""
    vk = np.sqrt(w.gm / rc)
    ref = -2.0 * w.stokes * (vk - eq_vtheta) / (1.0 + w.stokes ** 2)
    vr = E[5, 1:-1] / E[8, 1:-1]
    sel = (rc > 0.85) & (rc < 1.2)
    return (np.abs(vr[:, :, sel] - ref[sel]) / np.abs(ref[sel])).max()


def test_dust_settles_at_terminal_velocity():
    w = settling_workload()
    o = oracle.Oracle(w)
    E = oracle.initial_state(o)
    for _ in range(40):
        E = o.step(E, o.cfl_dt(E))
    assert o.take_status() == 0
    assert settling_error(w, E, o.coords(2)[0], o.coords(0)[0]) <= 1e-2


@pytest.mark.parametrize("stokes,steps", [(0.01, 400), (0.1, 400), (1.0, 2400)],
                         ids=["st_0.01", "st_0.1", "st_1"])
def test_dust_drifts_at_the_nsh_rate(stokes, steps):
    """Across the drift's maximum at St = 1 (the rate goes as St / (1 + St^2));
    each run covers several stopping times: 400 steps are ~1.8 time units,
    2400 ~10.6 (measured errors 0.74 %, 0.29 %, 0.52 %)."""
    w = replace(drift_workload(), stokes=stokes)
    o = oracle.Oracle(w)
    E = oracle.initial_state(o)
    for _ in range(steps):
        E = o.step(E, o.cfl_dt(E))
    assert o.take_status() == 0
    rc = o.coords(0)[0]
    vth = np.array([o.eq_prim(r, 0.0)[1] for r in rc])
    assert drift_error(w, E, rc, vth) <= 1e-2
