"""Pins of the Rossby-wave-instability workload (Sect. 4.3) as the oracle
builds it.

Sect. 4.3 puts a radial Gaussian bump, rho = rho0 (1 + delta G) with
G = exp(-((r - r0) / (sqrt(2) Delta_r))^2), on the equilibrium of App. A, and
seeds v_r = eps v_theta0 sin(m theta) G.  Here the bump belongs to the
equilibrium (rho and P scaled at the same temperature, v_theta0 in radial
balance with the bumped pressure).  The pins hold it to what fixes it from
outside the code: against the unbumped equilibrium the density ratio is
1 + delta G and the temperature is unchanged; the continuum radial and
vertical balances hold (finite differences of the oracle's own P(r, z),
which a dropped or sign-flipped bump term in v_theta0 fails); one step of the
bumped equilibrium leaves it unchanged (the balanced scheme of Sect. 2.8);
and the initial state departs from it only by the seed, whose projection
over theta is mode m alone with amplitude eps v_theta0 G.
"""
from dataclasses import replace
import math

import numpy as np

import oracle
import synthetic as syn

F_MU, F_MV, F_MW, F_EN, F_RHO = range(5)


def _prim(U, g):
    rho = U[F_RHO]
    u, v, ww = U[F_MU] / rho, U[F_MV] / rho, U[F_MW] / rho
    P = (g - 1.0) * (U[F_EN] - 0.5 * rho * (u * u + v * v + ww * ww))
    return rho, u, v, ww, P


def _bump(w, r):
    return np.exp(-((r - w.rwi_r0) / (math.sqrt(2.0) * w.rwi_width)) ** 2)


def test_bumped_equilibrium_against_the_plain_one():
    w = syn.scaled(syn.RWI, 24, 8, 16)
    ob, op = oracle.Oracle(w), oracle.Oracle(replace(w, rwi_delta=0.0))
    r, _ = ob.coords(0)
    rb, _, _, _, Pb = _prim(ob.equilibrium_state(), w.gamma)
    rp, _, _, _, Pp = _prim(op.equilibrium_state(), w.gamma)
    G = _bump(w, r)[None, None, :]
    np.testing.assert_allclose(rb / rp, np.broadcast_to(1.0 + w.rwi_delta * G, rb.shape), rtol=1e-14, atol=0)
    np.testing.assert_allclose(Pb / rb, Pp / rp, rtol=1e-13, atol=0)  # the temperature is kept
    assert np.abs(G - 1.0).min() < 0.02 and G.min() < 1e-10           # the grid spans the bump


def test_bumped_equilibrium_balances():
    """(1/rho) dP/dr = v_theta^2 / r - GM r / R^3 and (1/rho) dP/dz = -GM z / R^3,
    with v_theta inertial, by Richardson-extrapolated central differences of
    the oracle's P(r, z), where the bump's gradient is largest and away from it."""
    w = syn.scaled(syn.RWI, 8, 4, 4)
    o = oracle.Oracle(w)
    H = 0.05
    for r in (w.rwi_r0 - w.rwi_width, w.rwi_r0 - 0.3 * w.rwi_width, w.rwi_r0, w.rwi_r0 + w.rwi_width,
              w.rwi_r0 + 2.5 * w.rwi_width, 1.4):
        for z in (0.0, 0.7 * H, -1.6 * H):
            rho, vth, P = o.eq_prim(r, z)
            R3 = (r * r + z * z) ** 1.5

            def d(f, x, h):
                c1 = (f(x + h) - f(x - h)) / (2 * h)
                c2 = (f(x + h / 2) - f(x - h / 2)) / h
                return (4 * c2 - c1) / 3

            dPdr = d(lambda x: o.eq_prim(x, z)[2], r, 1e-3 * w.rwi_width)
            dPdz = d(lambda x: o.eq_prim(r, x)[2], z, 1e-3 * H)
            vin = vth  # eq_prim gives the inertial v_theta0
            lhs_r, rhs_r = dPdr / rho, vin * vin / r - w.gm * r / R3
            scale = w.gm / r ** 2
            assert abs(lhs_r - rhs_r) <= 1e-9 * scale, (r, z, lhs_r, rhs_r)
            assert abs(dPdz / rho + w.gm * z / R3) <= 1e-9 * scale, (r, z)
    # the bump's own term matters at this tolerance: without it the balance
    # is off by r T delta G'/(1 + delta G) / r, of order 1e-3 of GM / r^2
    r = w.rwi_r0 - w.rwi_width
    T = o.eq_prim(r, 0.0)[2] / o.eq_prim(r, 0.0)[0]
    G = _bump(w, r)
    dG = -(r - w.rwi_r0) / w.rwi_width ** 2 * G
    assert T * w.rwi_delta * dG / (1.0 + w.rwi_delta * G) > 1e3 * 1e-9 * w.gm / r ** 2


def test_bumped_equilibrium_is_stationary():
    """Two steps of the bumped equilibrium leave it unchanged (the balanced
    residual of Sect. 2.8 is taken on this equilibrium)."""
    w = syn.scaled(syn.RWI, 16, 8, 16)
    o = oracle.Oracle(w)
    E0 = o.equilibrium_state()
    E = E0.copy()
    for _ in range(2):
        E = o.step(E, o.cfl_dt(E))
    assert o.take_status() == 0
    np.testing.assert_allclose(E, E0, rtol=1e-13, atol=1e-15 * np.abs(E0).max())


def test_rwi_initial_state_is_equilibrium_plus_seed():
    w = syn.scaled(syn.RWI, 24, 48, 16)
    o = oracle.Oracle(w)
    E = oracle.initial_state(o)
    E0 = o.equilibrium_state()
    r, _ = o.coords(0)
    th, _ = o.coords(1)
    z, _ = o.coords(2)
    np.testing.assert_array_equal(E[[F_MV, F_MW, F_RHO]], E0[[F_MV, F_MW, F_RHO]])
    rho0 = E0[F_RHO]
    u = E[F_MU] / rho0
    np.testing.assert_allclose(E[F_EN] - E0[F_EN], 0.5 * rho0 * u * u, rtol=1e-6, atol=1e-15 * np.abs(E0[F_EN]).max())
    # the seed: mode m alone, amplitude eps v_theta0 G (inertial v_theta0):
    # the projection on sin(m theta) over the cell centres, and nothing left
    m = w.rwi_mode
    S = np.sin(m * th)[None, :, None]
    a = (2.0 / w.nth) * (u * S).sum(axis=1)
    vth0 = np.array([[o.eq_prim(ri, zk)[1] for ri in r] for zk in z])
    amp = w.rwi_eps * vth0 * _bump(w, r)[None, :]
    np.testing.assert_allclose(a, amp, rtol=1e-10, atol=1e-14 * amp.max())
    assert np.abs(u - a[:, None, :] * S).max() <= 1e-12 * amp.max()
