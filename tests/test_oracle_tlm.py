"""Pins of the oracle's tangent-linear mode against its own value map.

The tangent-linear step (dual numbers through the whole RK2 step, with the
star-pressure tangent taken from the implicit function theorem) must agree
with central differences of the plain FP64 step at a fixed dt.  That is a
check by the definition of the derivative, independent of how the tangent is
formed.  The limiter, the wave pattern of the Riemann solution and the dust
upwinding make the step piecewise smooth, so the states below are jittered
away from exact ties (an unperturbed disc has E' = 0 and minmod(0, 0) in every
cell) and directions are scaled to each cell's own deviation E' = E - E0: the
differences then cross a branch boundary in few cells only.
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle
import synthetic as syn
from tests.parity import jitter as _jitter


def _l1(a, b):
    return np.abs(a - b).sum(axis=(1, 2, 3)) / np.abs(b).sum(axis=(1, 2, 3))


def _central(o, E, d, dt, h):
    return (o.step(E + h * d, dt) - o.step(E - h * d, dt)) / (2.0 * h)


def test_tlm_values_are_the_step():
    w = syn.scaled(syn.VORTEX, 12, 10, 16)
    o = oracle.Oracle(w)
    E = oracle.initial_state(o)
    dt = o.cfl_dt(E)
    rng = np.random.default_rng(3)
    E1, _ = o.step_tlm(E, rng.standard_normal(E.shape), dt, dstokes=0.3)
    assert np.array_equal(E1, o.step(E, dt))


def test_tlm_zero_direction_gives_zero_tangent():
    w = syn.scaled(syn.VORTEX, 12, 10, 16)
    o = oracle.Oracle(w)
    E = oracle.initial_state(o)
    _, t = o.step_tlm(E, np.zeros_like(E), o.cfl_dt(E))
    assert not t.any()


@pytest.mark.parametrize("recon", [syn.RECON_CONSERVATIVE, syn.RECON_PRESSURE], ids=["conservative", "pressure"])
def test_tlm_disc_random_direction(recon):
    """Gas-only disc, every field of every cell perturbed at once (the paper's
    reconstruction and option 2, whose pressure departure and face energy
    carry their own tangents)."""
    w = replace(syn.scaled(syn.DISC_NOISE, 12, 10, 32), recon=recon)
    o = oracle.Oracle(w)
    rng = np.random.default_rng(1)
    E = _jitter(oracle.initial_state(o), w.gamma, rng, 1e-3)
    d = np.abs(E - o.equilibrium_state()) * rng.standard_normal(E.shape)
    dt = o.cfl_dt(E)
    _, t = o.step_tlm(E, d, dt)
    assert o.take_status() == 0
    # the best of two steps: larger ones cross limiter branches of the pressure
    # deviation (a conservative direction moves P' by O(Mach^2) more), smaller
    # ones lose digits to rounding
    err = min((_l1(_central(o, E, d, dt, h), t) for h in (1e-6, 3e-7)), key=lambda e: e.max())
    assert err.max() <= 1e-6, err


def test_tlm_sod_after_shock_formation():
    """Box with a shock, a contact and a rarefaction: every wave pattern of
    the exact solver (and the Newton tangent) is exercised."""
    w = syn.scaled(syn.SOD, 64, 2, 2)
    o = oracle.Oracle(w)
    rng = np.random.default_rng(1)
    E, _, _ = o.run(oracle.initial_state(o), steps=5)
    E = _jitter(E, w.gamma, rng, 1e-3)
    d = np.abs(E) * rng.standard_normal(E.shape)
    dt = o.cfl_dt(E)
    _, t = o.step_tlm(E, d, dt)
    err = _l1(_central(o, E, d, dt, 1e-7), t)
    assert err.max() <= 1e-6, err


@pytest.mark.parametrize("law", [0, 1])
def test_tlm_vortex_single_cells(law):
    """Bi-fluid vortex: one field of one cell at a time, every field, three
    interior cells; the 4-cell-deep stencil response must match."""
    w = replace(syn.scaled(syn.VORTEX, 12, 10, 32), drag_law=law)
    o = oracle.Oracle(w)
    rng = np.random.default_rng(1)
    E = _jitter(oracle.initial_state(o), w.gamma, rng, 1e-3)
    Ed = E - o.equilibrium_state()
    dt = o.cfl_dt(E)
    for f in range(9):
        for (k, j, i) in ((16, 5, 6), (28, 9, 10), (15, 0, 11)):
            d = np.zeros_like(E)
            d[f, k, j, i] = abs(Ed[f, k, j, i])
            _, t = o.step_tlm(E, d, dt)
            err = min(np.abs(_central(o, E, d, dt, h) - t).max() for h in (1e-4, 1e-5, 1e-6, 1e-7))
            assert err <= 1e-4 * np.abs(t).max(), (f, (k, j, i), err / np.abs(t).max())


@pytest.mark.parametrize("law", [0, 1])
def test_tlm_stokes_number(law):
    """d/dSt of the step: the drag exchange moves the dust momenta first."""
    w = replace(syn.scaled(syn.VORTEX, 12, 10, 32), drag_law=law)
    o = oracle.Oracle(w)
    rng = np.random.default_rng(2)
    E = _jitter(oracle.initial_state(o), w.gamma, rng, 1e-3)
    dt = o.cfl_dt(E)
    _, t = o.step_tlm(E, np.zeros_like(E), dt, dstokes=1.0)
    h = 1e-5 * w.stokes
    fd = (o.step_tlm(E, 0 * E, dt, stokes=w.stokes + h)[0] - o.step_tlm(E, 0 * E, dt, stokes=w.stokes - h)[0]) / (2 * h)
    err = _l1(fd, t)
    # the dust momenta and the small gas momenta (radial, vertical) carry the
    # exchange; the azimuthal gas momentum, energy and densities respond at
    # second hand, below the rounding of the difference quotient
    assert err[[0, 2, 5, 6, 7]].max() <= 1e-5, err
