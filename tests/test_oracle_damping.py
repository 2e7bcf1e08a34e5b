"""Pins of the oracle's wave-killing zones (Sect. 2.4, reading R17).

The paper names radial wave-killing boundaries without writing them down; the
oracle takes the relaxation of de Val-Borro et al. (2006): inside a zone at
each radial edge, dE'/dt = -E' R(r) / tau for the gas departures, with R the
parabola that is 1 at the domain boundary and 0 (with zero slope) at the
zone's edge, and tau the Keplerian orbital period at that boundary.  Parity
for the profile and the constants is unpinned (they come from the cited work,
not the paper); the pins check what the term must be whatever its constants:
local in the cell, linear in E', one rate for the five gas fields, none for
dust, zero in the interior, and a rate whose radial profile is a parabola
through its end conditions with 1/tau = Omega_K / (2 pi) at the boundary.
"""
import numpy as np
import pytest

import oracle
import synthetic as syn
from tests.parity import jitter

R_IN, R_OUT = 0.5, 2.0
EIN, EOUT = 1.25 * R_IN, 0.84 * R_OUT


def _damping_part(o, E, f=0.01):
    """G with the zones minus G without; a short period (f = 0.01) lifts the
    term well above the rounding of the two right-hand sides."""
    o.set_damping(EIN, EOUT, f)
    on = o.rhs(E)
    o.set_damping(EIN, EOUT, 0.0)
    off = o.rhs(E)
    assert o.take_status() == 0
    return on - off


def _noisy(o, rng):
    """Jittered initial state (grids of 16 or more z cells: coarser ones put
    jittered face pressures of the thin, cold disc edges below zero)."""
    return jitter(oracle.initial_state(o), o.w.gamma, rng, 1e-3)


@pytest.mark.parametrize("base", ["vortex", "disc"])
def test_local_linear_gas_only(base):
    w = syn.scaled(syn.VORTEX if base == "vortex" else syn.DISC_NOISE, 48, 6, 16)
    o = oracle.Oracle(w)
    E = _noisy(o, np.random.default_rng(1))
    Ed = E - o.equilibrium_state()
    D = _damping_part(o, E)
    r = o.coords(0)[0]
    inside = (r >= EIN) & (r <= EOUT)
    assert not D[..., inside].any()              # interior untouched
    assert not D[5:].any()                       # dust untouched
    V = o.volumes()[None, None, :]
    k = -D[:5] / (V * Ed[:5])                    # rate per field and cell
    zone = ~inside
    # one rate for all five gas fields, the same in every theta and z
    # (to the rounding of G_on - G_off)
    ref = k[4][..., zone]
    assert np.allclose(k[..., zone], ref[None], rtol=1e-8, atol=0)
    assert np.allclose(ref, ref[:1, :1], rtol=1e-9, atol=0)
    # linear: doubling the departure doubles the term
    D2 = _damping_part(o, o.equilibrium_state() + 2.0 * Ed)
    assert np.allclose(D2[:5], 2.0 * D[:5], rtol=1e-8, atol=0)
    # the period factor divides the rate
    D3 = _damping_part(o, E, f=0.04)
    assert np.allclose(D3[:5], 0.25 * D[:5], rtol=1e-8, atol=0)


def test_rate_profile_is_the_boundary_parabola():
    """Fit a quadratic to the per-cell rates of each zone (fine radial grid):
    zero with zero slope at the zone's edge, Omega_K / (2 pi) at the domain
    boundary."""
    w = syn.scaled(syn.DISC_NOISE, 400, 4, 16)
    o = oracle.Oracle(w)
    E = _noisy(o, np.random.default_rng(2))
    Ed = E - o.equilibrium_state()
    D = _damping_part(o, E)
    r = o.coords(0)[0]
    k = (-D[4] / (o.volumes()[None, None, :] * Ed[4]))[0, 0]
    for lo, hi, edge, bound in ((R_IN, EIN, EIN, R_IN), (EOUT, R_OUT, EOUT, R_OUT)):
        sel = (r > lo) & (r < hi)
        c = np.polyfit(r[sel] - edge, k[sel], 2)
        assert abs(c[2]) <= 1e-10 * c[0] and abs(c[1]) <= 1e-9 * c[0] * abs(bound - edge), c
        at_bound = np.polyval(c, bound - edge)  # f = 0.01: tau is a hundredth of the period
        assert at_bound == pytest.approx(np.sqrt(w.gm / bound ** 3) / (2 * np.pi) / 0.01, rel=1e-10)


def test_equilibrium_stays_bit_exact_with_damping():
    w = syn.scaled(syn.DISC_NOISE, 24, 8, 16)
    o = oracle.Oracle(w)
    o.set_damping(EIN, EOUT)
    E = o.equilibrium_state()
    dt = o.cfl_dt(E)
    assert np.array_equal(o.step(o.step(E, dt), dt), E)


def test_zones_calm_the_edges():
    """Over 40 steps of the noisy disc (tau a hundredth of the period) the
    zones remove departure mass at the radial edges and leave the middle of
    the disc as it was."""
    w = syn.scaled(syn.DISC_NOISE, 32, 8, 32)
    o = oracle.Oracle(w)
    E0 = oracle.initial_state(o)
    Eq = o.equilibrium_state()
    V = o.volumes()[None, None, :]
    r = o.coords(0)[0]
    zone, mid = (r < EIN) | (r > EOUT), (r > 0.9) & (r < 1.3)
    runs = {}
    for f in (0.0, 0.01):
        o.set_damping(EIN, EOUT, f)
        E, _, dts = o.run(E0.copy(), steps=40) if f == 0.0 else o.run(E0.copy(), dts=runs[0.0][1])
        assert o.take_status() == 0
        runs[f] = (np.abs((E - Eq)[4]) * V, dts)
    a, b = runs[0.0][0], runs[0.01][0]
    assert b[..., zone].sum() < 0.8 * a[..., zone].sum()  # measured 0.70
    # the middle of the disc has hardly heard of the zones yet: its departure
    # mass moves by ~3e-8 of itself (numerical signal through the stencil's
    # domain of dependence), against 30 % in the zones
    assert abs(b[..., mid].sum() - a[..., mid].sum()) <= 1e-6 * a[..., mid].sum()


def test_bad_zones_are_refused():
    o = oracle.Oracle(syn.scaled(syn.DISC_NOISE, 24, 8, 16))
    for ein, eout in ((0.4, 1.6), (0.6, 2.5), (1.5, 1.0)):
        with pytest.raises(ValueError):
            o.set_damping(ein, eout)
    box = oracle.Oracle(syn.scaled(syn.SOD, 16, 2, 2))
    with pytest.raises(ValueError):
        box.set_damping(0.2, 0.8)


def test_tlm_carries_the_damping():
    """Tangent-linear step with the zones on against central differences
    (the gas-only disc and direction of the plain tangent-linear pin)."""
    w = syn.scaled(syn.DISC_NOISE, 12, 10, 32)
    o = oracle.Oracle(w)
    o.set_damping(EIN, EOUT, 0.05)
    rng = np.random.default_rng(1)
    E = _noisy(o, rng)
    d = np.abs(E - o.equilibrium_state()) * rng.standard_normal(E.shape)
    dt = o.cfl_dt(E)
    _, t = o.step_tlm(E, d, dt)
    assert o.take_status() == 0
    err = min((np.abs((o.step(E + h * d, dt) - o.step(E - h * d, dt)) / (2 * h) - t).sum(axis=(1, 2, 3))
               / np.abs(t).sum(axis=(1, 2, 3)) for h in (1e-6, 3e-7)), key=lambda e: e.max())
    assert err.max() <= 1e-6, err
