"""Pins of the Rossby-wave-instability workload's initial state (Sect. 4.3)
as the oracle builds it.

Sect. 4.3 puts a radial Gaussian bump, rho = rho0 (1 + delta G) with
G = exp(-((r - r0) / (sqrt(2) Delta_r))^2), on the equilibrium of App. A, and
seeds v_r = eps v_theta0 sin(m theta) G.  The pins read the state back: the
density ratio is 1 + delta G at every cell, the temperature P / rho and the
azimuthal velocity are the equilibrium's, v_z = 0, and over theta the radial
velocity holds the sine of mode m alone, with amplitude eps v_theta0 G
(v_theta0 from App. A's equilibrium in the inertial frame).
"""
import math

import numpy as np

import oracle
import synthetic as syn

F_MU, F_MV, F_MW, F_EN, F_RHO = range(5)


def test_rwi_initial_state():
    w = syn.scaled(syn.RWI, 24, 48, 16)
    o = oracle.Oracle(w)
    E = oracle.initial_state(o)
    E0 = o.equilibrium_state()
    r, _ = o.coords(0)
    th, _ = o.coords(1)
    z, _ = o.coords(2)
    g = w.gamma
    G = np.exp(-((r - w.rwi_r0) / (math.sqrt(2.0) * w.rwi_width)) ** 2)
    assert np.allclose(E[F_RHO] / E0[F_RHO], 1.0 + w.rwi_delta * G[None, None, :], rtol=1e-14, atol=0)

    def prim(U):
        rho = U[F_RHO]
        u, v, ww = U[F_MU] / rho, U[F_MV] / rho, U[F_MW] / rho
        P = (g - 1.0) * (U[F_EN] - 0.5 * rho * (u * u + v * v + ww * ww))
        return rho, u, v, ww, P

    rho, u, v, ww, P = prim(E)
    rho0, _, v0, _, P0 = prim(E0)
    assert np.allclose(P / rho, P0 / rho0, rtol=1e-12, atol=0)      # the equilibrium temperature
    assert not ww.any()                                             # no v_z
    # radial balance of the bump: v_theta^2 = v_theta0^2 + r T delta G' / (1 + delta G), inertial speeds
    R = r[None, None, :]
    dG = -(R - w.rwi_r0) / w.rwi_width ** 2 * G[None, None, :]
    vin, vin0 = v + w.omega_frame * R, v0 + w.omega_frame * R
    np.testing.assert_allclose(vin ** 2 - vin0 ** 2, R * (P0 / rho0) * w.rwi_delta * dG / (1.0 + w.rwi_delta * G),
                               rtol=1e-8, atol=1e-12 * (vin0 ** 2).max())
    # the seed: mode m alone, amplitude eps v_theta0 G (inertial v_theta0):
    # the projection on sin(m theta) over the cell centres, and nothing left
    m = w.rwi_mode
    S = np.sin(m * th)[None, :, None]
    a = (2.0 / w.nth) * (u * S).sum(axis=1)
    vth0 = np.array([[o.eq_prim(ri, zk)[1] for ri in r] for zk in z])
    amp = w.rwi_eps * vth0 * G[None, :]
    np.testing.assert_allclose(a, amp, rtol=1e-10, atol=1e-14 * amp.max())
    assert np.abs(u - a[:, None, :] * S).max() <= 1e-12 * amp.max()
