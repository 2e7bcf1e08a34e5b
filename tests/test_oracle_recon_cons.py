"""Pins of the oracle's reconstruction of the conservative departures
(Sect. 2.7 on the conservative variables of App. B), the default mode.

Sect. 2.7 writes each face state as the equilibrium at the face plus a
parabola through the departures E'_p = E_p - E0_p of the three cells, for
each conservative variable p separately.  So a state whose departures are, in
every variable, the same quadratic function of the coordinate along one axis
(with the limiter left alone: monotone, gentle curvature) has face states
E0(face) + that quadratic at the face coordinate, exactly up to rounding, on
the logarithmic radial mesh as on the uniform theta and z meshes.  The
primitive option, which interpolates the departures of (rho, u, v, w, P),
does not reproduce such a profile: the test tells the two readings apart, so
a reconstruction silently switched to primitive variables fails it.
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle
import synthetic as syn


def _setup(ax, recon):
    w = replace(syn.scaled(syn.DISC_NOISE, 16, 16, 16), recon=recon)
    o = oracle.Oracle(w)
    E0 = o.equilibrium_state()
    xc = o.coords(ax)[0]
    x0, span = xc[0], xc[-1] - xc[0]
    # per-variable amplitudes: 1e-4 of the midplane equilibrium magnitude of
    # each variable (the radial and vertical momenta use the azimuthal one)
    k_mid = w.nz // 2
    scale = np.abs(E0[:, k_mid]).max(axis=(1, 2))
    scale[[syn.F_MU, syn.F_MW]] = scale[syn.F_MV]
    amp = 1e-4 * scale
    s = (xc - x0) / span + 0.7                      # in [0.7, 1.7]: monotone quadratic below
    prof = s + 0.15 * s * s
    shape = [1, 1, 1]
    shape[2 - ax] = len(xc)                          # (nz, nth, nr) axis order
    q = prof.reshape(shape)
    E = E0 + amp[:, None, None, None] * q[None]
    return w, o, E, amp, x0, span


def _quad_at(x, amp, x0, span):
    s = (x - x0) / span + 0.7
    return amp * (s + 0.15 * s * s)


@pytest.mark.parametrize("ax", [0, 1, 2])
def test_conservative_quadratic_departure_is_exact(ax):
    w, o, E, amp, x0, span = _setup(ax, syn.RECON_CONSERVATIVE)
    xf = o.coords(ax)[1]
    Eq = o.equilibrium_state()
    k_mid, j = w.nz // 2, 3
    n = (w.nr, w.nth, w.nz)[ax]
    checked = 0
    for c in range(2, n - 2):
        cell = [6, j, k_mid]
        cell[ax] = c
        if ax == 2 and abs(c - k_mid) > 3:
            continue
        Um, Up = o.recon_faces(E, ax, *cell)
        Qm, Qp = o.recon_faces(Eq, ax, *cell)   # E0 on the two faces (zero departure)
        for U, Q, xface in ((Um, Qm, xf[c]), (Up, Qp, xf[c + 1])):
            want = _quad_at(xface, amp, x0, span)
            got = U[:5] - Q[:5]
            assert np.allclose(got, want, rtol=1e-10, atol=1e-13 * np.abs(Q[:5]).max()), (ax, c, got, want)
        checked += 1
    assert checked >= 4


@pytest.mark.parametrize("ax", [0, 2])
def test_primitive_option_differs(ax):
    """The same state under the primitive option gives face states that miss the
    conservative quadratic by far more than rounding (so the default's pin is
    not vacuous)."""
    w, o, E, amp, x0, span = _setup(ax, syn.RECON_PRIMITIVE)
    xf = o.coords(ax)[1]
    Eq = o.equilibrium_state()
    k_mid = w.nz // 2
    worst = 0.0
    for c in range(2, 6):
        cell = [6, 3, k_mid]
        cell[ax] = c if ax == 0 else k_mid - 2 + c % 4
        Um, _ = o.recon_faces(E, ax, *cell)
        Qm, _ = o.recon_faces(Eq, ax, *cell)
        want = _quad_at(xf[cell[ax]], amp, x0, span)
        worst = max(worst, float(np.max(np.abs(Um[:5] - Qm[:5] - want) / np.abs(amp))))
    assert worst > 1e-6, worst


def test_equilibrium_faces_are_the_face_equilibrium():
    """Zero departure: each face state is E0 evaluated at the face (App. A at
    the face coordinate), here checked on r faces against the equilibrium
    primitives the oracle evaluates at (r_face, z)."""
    w = syn.scaled(syn.DISC_NOISE, 16, 8, 16)
    o = oracle.Oracle(w)
    Eq = o.equilibrium_state()
    rf = o.coords(0)[1]
    z = o.coords(2)[0]
    for i in (3, 8, 12):
        Um, Up = o.recon_faces(Eq, 0, i, 2, 5)
        for U, r in ((Um, rf[i]), (Up, rf[i + 1])):
            rho, vth, p = o.eq_prim(r, z[5])
            v = vth - w.omega_frame * r
            want = np.array([0.0, rho * v, 0.0, 0.5 * rho * v * v + p / (w.gamma - 1.0), rho])
            assert np.allclose(U[:5], want, rtol=1e-14, atol=1e-300)
