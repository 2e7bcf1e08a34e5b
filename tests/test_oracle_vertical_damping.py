"""Pins of the oracle's vertical sheared damped boundary (Sect. 2.4, reading
R21).

Sect. 2.4 names, after the works it cites, a "sheared damped" boundary for
the vertical direction without a formula.  The oracle reads it as the
equilibrium (sheared Keplerian) ghost cells of Sect. 2.4 plus a relaxation of
the gas departures towards the equilibrium in |z| > z_e, the radial
wave-killing form of R17 turned vertical: rate R(z) / tau(r), R the parabola
that is 1 at |z| = z_max and 0 with zero slope at z_e, tau = f x the local
Keplerian orbital period.  Parity for the profile and the constants is
unpinned; the pins check the structure: local, linear, one rate for the five
gas fields, none for dust, zero for |z| <= z_e, mirror symmetric in z, a
parabola through its end conditions with 1/tau = Omega_K(r) / (2 pi f) at the
boundary (Omega_K from Kepler's law in the test), additive with the radial
zones, an undisturbed disc kept bit for bit, and the tangent-linear step
against central differences.
"""
import math

import numpy as np
import pytest

import oracle
import synthetic as syn
from tests.parity import jitter

ZE = 0.06          # zone edge (the domain is |z| <= 0.15)
F = 0.01           # tau = F x the local orbital period: far above rounding


def _part(o, E):
    o.set_vertical_damping(ZE, F)
    on = o.rhs(E)
    o.set_vertical_damping(ZE, 0.0)
    off = o.rhs(E)
    assert o.take_status() == 0
    return on - off


@pytest.mark.parametrize("base", ["vortex", "disc"])
def test_local_linear_gas_only(base):
    w = syn.scaled(syn.VORTEX if base == "vortex" else syn.DISC_NOISE, 16, 6, 32)
    o = oracle.Oracle(w)
    E = jitter(oracle.initial_state(o), w.gamma, np.random.default_rng(3), 1e-3)
    Ed = E - o.equilibrium_state()
    D = _part(o, E)
    z = o.coords(2)[0]
    inside = np.abs(z) <= ZE
    assert not D[:, inside].any() and not D[5:].any()
    V = o.volumes()[None, None, :]
    k = -D[:5] / (V * Ed[:5])
    ref = k[4][~inside]
    assert np.allclose(k[:, ~inside], ref[None], rtol=1e-7, atol=0)        # one rate for the gas fields
    assert np.allclose(ref, ref[:, :1, :], rtol=1e-9, atol=0)              # the same in every theta


def test_profile_symmetry_and_period():
    w = syn.scaled(syn.DISC_NOISE, 8, 4, 64)
    o = oracle.Oracle(w)
    o.set_vertical_damping(ZE, F)
    z = o.coords(2)[0]
    r = o.coords(0)[0]
    zmax = w.x1[2]
    for i in range(w.nr):
        rate = np.array([o.damping_rate(i, k) for k in range(w.nz)])
        assert np.allclose(rate, rate[::-1], rtol=1e-12, atol=0)             # mirror symmetric
        assert not rate[np.abs(z) <= ZE].any()
        up = z > ZE
        c = np.polyfit(z[up], rate[up], 2)                                   # an exact quadratic in z
        assert np.allclose(np.polyval(c, z[up]), rate[up], rtol=1e-10, atol=0)
        omk = math.sqrt(w.gm / r[i] ** 3)
        assert np.polyval(c, zmax) == pytest.approx(omk / (2 * math.pi * F), rel=1e-9)
        assert abs(np.polyval(c, ZE)) <= 1e-9 * np.polyval(c, zmax)          # 0 at the edge ...
        assert abs(np.polyval(np.polyder(c), ZE)) <= 1e-8 * np.polyval(c, zmax) / (zmax - ZE)  # ... zero slope


def test_adds_to_the_radial_zones():
    w = syn.scaled(syn.DISC_NOISE, 32, 4, 32)
    o = oracle.Oracle(w)
    ez = (0.625, 1.68)
    o.set_damping(*ez, 0.02)
    radial = np.array([[o.damping_rate(i, k) for i in range(w.nr)] for k in range(w.nz)])
    o.set_vertical_damping(ZE, F)
    both = np.array([[o.damping_rate(i, k) for i in range(w.nr)] for k in range(w.nz)])
    o.set_damping(*ez, 0.0)
    vertical = np.array([[o.damping_rate(i, k) for i in range(w.nr)] for k in range(w.nz)])
    assert radial.any() and vertical.any()
    assert np.allclose(both, radial + vertical, rtol=1e-15, atol=0)


def test_equilibrium_bit_exact():
    w = syn.scaled(syn.VORTEX, 16, 8, 32)
    o = oracle.Oracle(w)
    o.set_vertical_damping(ZE, F)
    E0 = o.equilibrium_state()
    E, _, _ = o.run(E0.copy(), steps=5)
    assert np.array_equal(E, E0)


def test_tangent_linear_step():
    w = syn.scaled(syn.VORTEX, 16, 8, 32)
    o = oracle.Oracle(w)
    o.set_vertical_damping(ZE, F)
    rng = np.random.default_rng(4)
    E = jitter(oracle.initial_state(o), w.gamma, rng, 1e-3)
    d = jitter(E, w.gamma, rng, 1e-3) - E
    dt = o.cfl_dt(E)
    _, t = o.step_tlm(E, d, dt)
    err = min(np.abs((o.step(E + h * d, dt) - o.step(E - h * d, dt)) / (2 * h) - t).sum() / np.abs(t).sum()
              for h in (1e-5, 1e-6))
    assert err <= 1e-6, err


def test_bad_zones_are_refused():
    o = oracle.Oracle(syn.scaled(syn.DISC_NOISE, 8, 4, 8))
    for ze in (-0.01, 0.16, 0.2):
        with pytest.raises(ValueError):
            o.set_vertical_damping(ze, 1.0)
    o.set_vertical_damping(0.1, 0.0)  # off is always accepted
