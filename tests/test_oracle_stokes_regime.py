"""Pins of the oracle's Stokes drag regime (Sect. 2.9, drag law 2, reading R19).

Sect. 2.9 gives the stopping time in two regimes: Epstein, t_E = rho_s r_p /
(rho_g c_s), while the particle radius is at most 9/4 of the gas mean free
path lambda ~ 1/rho_g, and Stokes, t_S = (4/9)(r_p / lambda) t_E, above.  With
kappa = r_p / lambda_0 (lambda = lambda_0 / rho_g) the switch sits at
kappa rho_g = 9/4.  The pins read the stopping time back from the oracle's
semi-implicit drag (the relative velocity relaxes by 1 + tau (1 + eps) / t_s
in one stage) and check the law's own properties: law 2 is law 1 below the
switch, the two meet at the switch, above it t_s is (4/9) kappa rho_g times
the Epstein value and no longer depends on the gas density (at a fixed sound
speed), and the tangent-linear step agrees with central differences.
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle
import synthetic as syn
from tests.parity import jitter


def _stopping_time(o, U, tau, i=3):
    """t_s from one drag call: dv_new = dv / (1 + tau (1 + eps) / t_s)."""
    out = o.drag(i, U, tau)
    dv0 = U[6] / U[8] - U[1] / U[4]
    dv1 = out[6] / out[8] - out[1] / out[4]
    eps = U[8] / U[4]
    return tau * (1.0 + eps) / (dv0 / dv1 - 1.0)


def _cell(rho, c2=1e-3, gamma=1.4):
    """Gas at density rho with P = c2 rho (fixed sound speed), dust at 1e-2 rho
    moving 1e-3 faster azimuthally."""
    U = np.zeros(9)
    U[4] = rho
    U[1] = rho * 0.1
    U[3] = c2 * rho / (gamma - 1.0) + 0.5 * rho * 0.1 ** 2
    U[8] = 1e-2 * rho
    U[6] = U[8] * 0.101
    return U


def _oracle(law, kappa):
    w = replace(syn.scaled(syn.VORTEX, 12, 10, 16), drag_law=law)
    o = oracle.Oracle(w)
    o.set_stokes_regime(kappa)
    return o


def test_law_two_is_epstein_below_the_switch():
    o1, o2 = _oracle(1, 0.0), _oracle(2, 1.0)
    for rho in (0.1, 1.0, 2.2):  # kappa rho < 9/4
        U = _cell(rho)
        assert np.array_equal(o1.drag(3, U, 1e-3), o2.drag(3, U, 1e-3))


def test_stokes_factor_and_continuity_at_the_switch():
    o1, o2 = _oracle(1, 0.0), _oracle(2, 1.0)
    for rho in (2.25 * (1 + 1e-9), 3.0, 10.0, 50.0):
        U = _cell(rho)
        tE, tS = _stopping_time(o1, U, 1e-3), _stopping_time(o2, U, 1e-3)
        assert tS / tE == pytest.approx((4.0 / 9.0) * rho, rel=1e-8), rho
    # the two laws meet at the switch
    U = _cell(2.25 * (1 + 1e-9))
    assert _stopping_time(o2, U, 1e-3) == pytest.approx(_stopping_time(o1, U, 1e-3), rel=1e-8)


def test_stokes_stopping_time_does_not_depend_on_the_gas_density():
    """t_S = (4/9) kappa rho_s r_p / c_s: in the Stokes regime the density
    cancels (at a fixed sound speed), while the Epstein time falls as 1/rho."""
    o1, o2 = _oracle(1, 0.0), _oracle(2, 1.0)
    tS = [_stopping_time(o2, _cell(rho), 1e-3) for rho in (4.0, 12.0, 36.0)]
    tE = [_stopping_time(o1, _cell(rho), 1e-3) for rho in (4.0, 12.0, 36.0)]
    assert np.allclose(tS, tS[0], rtol=1e-8)
    assert tE[0] / tE[1] == pytest.approx(3.0, rel=1e-8) and tE[1] / tE[2] == pytest.approx(3.0, rel=1e-8)


def test_tlm_with_the_stokes_regime():
    """The switch splits the disc (kappa puts about half of the cells in the
    Stokes regime).  As in the plain tangent-linear pin, one field of one cell
    at a time, in cells well inside each regime: the tangent-linear step
    against central differences (best of four steps, <= 1e-4 of its largest
    entry)."""
    w = replace(syn.scaled(syn.VORTEX, 12, 10, 16), drag_law=2)
    o = oracle.Oracle(w)
    rng = np.random.default_rng(7)
    E = jitter(oracle.initial_state(o), w.gamma, rng, 1e-3)
    Ed = E - o.equilibrium_state()
    kappa = 2.25 / np.median(E[4])
    o.set_stokes_regime(kappa)
    x = kappa * E[4]
    assert 0.2 < (x > 2.25).mean() < 0.8
    dt = o.cfl_dt(E)
    picks = []
    for regime in (x > 2.25 * 1.2, x < 2.25 / 1.2):
        k, j, i = np.nonzero(regime & (np.arange(w.nr)[None, None, :] >= 3) & (np.arange(w.nr)[None, None, :] < 9))
        picks += [(k[q], j[q], i[q]) for q in rng.choice(len(k), 2, replace=False)]
    for (k, j, i) in picks:
        for f in (4, 8, 6):  # gas density, dust density, dust azimuthal momentum
            d = np.zeros_like(E)
            d[f, k, j, i] = abs(Ed[f, k, j, i]) + 1e-3 * abs(E[f, k, j, i])
            _, t = o.step_tlm(E, d, dt)
            err = min(np.abs((o.step(E + h * d, dt) - o.step(E - h * d, dt)) / (2 * h) - t).max()
                      for h in (1e-4, 1e-5, 1e-6, 1e-7))
            assert err <= 1e-4 * np.abs(t).max(), (f, (k, j, i), x[k, j, i], err / np.abs(t).max())
    assert o.take_status() == 0
