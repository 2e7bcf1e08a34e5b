"""Pins of option 2 of the oracle's reconstruction (reading R2): the
parabola and MinMod of Sect. 2.7 on the departures of rho, rho u, rho v,
rho w and of the pressure P(E) - P(E0), the face energy following from the
face pressure, momenta and density.

A state whose density, momentum and pressure departures are the same
quadratic function of the coordinate along one axis (limiter left alone)
then has face states whose density, momenta and pressure are the face
equilibrium's plus that quadratic at the face coordinate, exactly up to
rounding, and whose energy is P / (gamma - 1) + |m|^2 / (2 rho) of those.
The paper's mode (the energy departure interpolated instead) misses the
face pressure of such a state, so the pin tells the two apart.
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle
import synthetic as syn

MU, MV, MW, EN, RHO = range(5)


def _pressure(g, U):
    return (g - 1.0) * (U[EN] - 0.5 * (U[MU] ** 2 + U[MV] ** 2 + U[MW] ** 2) / U[RHO])


def _setup(ax, recon):
    w = replace(syn.scaled(syn.DISC_NOISE, 16, 16, 16), recon=recon)
    o = oracle.Oracle(w)
    E0 = o.equilibrium_state()
    g = w.gamma
    xc = o.coords(ax)[0]
    x0, span = xc[0], xc[-1] - xc[0]
    k_mid = w.nz // 2
    scale = np.abs(E0[:, k_mid]).max(axis=(1, 2))
    scale[[MU, MW]] = scale[MV]
    P0 = _pressure(g, E0)
    amp = 1e-4 * scale
    amp_p = 1e-4 * np.abs(P0[k_mid]).max()
    s = (xc - x0) / span + 0.7
    prof = s + 0.15 * s * s
    shape = [1, 1, 1]
    shape[2 - ax] = len(xc)
    q = prof.reshape(shape)
    E = E0.copy()
    for f in (MU, MV, MW, RHO):
        E[f] = E0[f] + amp[f] * q
    P = P0 + amp_p * q
    E[EN] = P / (g - 1.0) + 0.5 * (E[MU] ** 2 + E[MV] ** 2 + E[MW] ** 2) / E[RHO]
    return w, o, E, amp, amp_p, x0, span


def _quad(x, x0, span):
    s = (x - x0) / span + 0.7
    return s + 0.15 * s * s


def _faces(w, o, E, ax):
    """(face coordinate, reconstructed state, equilibrium face state) of the
    lower faces of interior cells along ax."""
    xf = o.coords(ax)[1]
    k_mid, j = w.nz // 2, 3
    n = (w.nr, w.nth, w.nz)[ax]
    out = []
    for c in range(2, n - 2):
        cell = [6, j, k_mid]
        cell[ax] = c
        Um, _ = o.recon_faces(E, ax, *cell)
        U0m, _ = o.recon_faces(o.equilibrium_state(), ax, *cell)
        out.append((xf[c], Um, U0m))
    return out


@pytest.mark.parametrize("ax", [0, 1, 2])
def test_pressure_option_quadratic_is_exact(ax):
    w, o, E, amp, amp_p, x0, span = _setup(ax, syn.RECON_PRESSURE)
    g = w.gamma
    for x, Um, U0m in _faces(w, o, E, ax):
        qq = _quad(x, x0, span)
        for f in (MU, MV, MW, RHO):
            assert abs(Um[f] - (U0m[f] + amp[f] * qq)) <= 1e-12 * max(abs(U0m[f]), amp[f]), (ax, f)
        P = _pressure(g, Um)
        P0 = _pressure(g, U0m)
        assert abs(P - (P0 + amp_p * qq)) <= 1e-10 * amp_p, (ax, P - P0, amp_p * qq)


def test_the_paper_mode_misses_that_face_pressure():
    ax = 0
    w, o, E, amp, amp_p, x0, span = _setup(ax, syn.RECON_CONSERVATIVE)
    errs = []
    for x, Um, U0m in _faces(w, o, E, ax):
        errs.append(abs(_pressure(w.gamma, Um) - _pressure(w.gamma, U0m) - amp_p * _quad(x, x0, span)) / amp_p)
    assert max(errs) > 1e-6, max(errs)
