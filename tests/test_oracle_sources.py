"""Pins of the oracle's App. B source vector against the effective potential.

In the rotating frame (reading R6) the star's gravity (Sect. 2.1) and the
centrifugal force derive from one scalar, Phi_eff = -GM / sqrt(r^2 + z^2) -
Omega_f^2 r^2 / 2.  The test differentiates that scalar by central
differences, independently of the oracle's closed-form forces, and checks on
random gas and dust states at several cells:
- the vertical momentum source is -rho dPhi/dz;
- the energy source is the work of that force, -rho (u dPhi/dr + w dPhi/dz),
  so it cannot depend on the azimuthal velocity (the Coriolis force does no
  work);
- the radial momentum source, less the geometric terms rho v^2 / r + P / r
  and the Coriolis term 2 Omega_f rho v, is -rho dPhi/dr;
- the dust momentum sources are the same without pressure, and no mass
  source appears.
A dropped or sign-flipped gravity, centrifugal or work term fails one of
these.
"""
import numpy as np
import pytest

import oracle
import synthetic as syn

MU, MV, MW, EN, RHO, DMU, DMV, DMW, DRHO = range(9)


def _phi(w, r, z):
    return -w.gm / np.sqrt(r * r + z * z) - 0.5 * w.omega_frame ** 2 * r * r


def _grad(w, r, z, h=1e-5):
    dr = (_phi(w, r + h, z) - _phi(w, r - h, z)) / (2 * h)
    dz = (_phi(w, r, z + h) - _phi(w, r, z - h)) / (2 * h)
    return dr, dz


def _state(rng, g):
    rho, rd = rng.uniform(0.5, 2.0), rng.uniform(0.01, 0.1)
    u, v, w = rng.uniform(-0.3, 0.3, 3)
    ud, vd, wd = rng.uniform(-0.3, 0.3, 3)
    P = rng.uniform(0.1, 1.0)
    U = np.array([rho * u, rho * v, rho * w, P / (g - 1) + 0.5 * rho * (u * u + v * v + w * w), rho,
                  rd * ud, rd * vd, rd * wd, rd])
    return U, (rho, u, v, w, P, rd, ud, vd, wd)


@pytest.mark.parametrize("omega", [1.0, 0.0, 0.63])
def test_sources_follow_the_effective_potential(omega):
    from dataclasses import replace
    w = replace(syn.scaled(syn.VORTEX, 12, 8, 16), omega_frame=omega)
    o = oracle.Oracle(w)
    rc, _ = o.coords(0)
    zc, _ = o.coords(2)
    rng = np.random.default_rng(11)
    for (i, k) in ((0, 0), (5, 3), (11, 15), (7, 8)):
        r, z = rc[i], zc[k]
        pr, pz = _grad(w, r, z)
        for _ in range(3):
            U, (rho, u, v, ww, P, rd, ud, vd, wd) = _state(rng, w.gamma)
            S = o.sources(i, 2, k, U)
            scale = rho * (abs(pr) + abs(pz)) + P / r
            assert S[RHO] == 0.0 and S[DRHO] == 0.0
            assert S[MW] == pytest.approx(-rho * pz, abs=1e-8 * scale)
            assert S[EN] == pytest.approx(-rho * (u * pr + ww * pz), abs=1e-8 * scale)
            radial = S[MU] - (rho * v * v / r + P / r + 2 * omega * rho * v)
            assert radial == pytest.approx(-rho * pr, abs=1e-8 * scale)
            assert S[DMW] == pytest.approx(-rd * pz, abs=1e-8 * scale)
            assert S[DMU] - (rd * vd * vd / r + 2 * omega * rd * vd) == pytest.approx(-rd * pr, abs=1e-8 * scale)
            # the Coriolis force does no work: the energy source ignores v
            U2 = U.copy()
            U2[MV] += rho * 0.2
            U2[EN] += 0.5 * rho * ((v + 0.2) ** 2 - v * v)
            assert o.sources(i, 2, k, U2)[EN] == S[EN]


def test_rotating_frame_sources_are_the_inertial_ones():
    """The same gas seen from a frame rotating at Omega_f: with v_in = v +
    Omega_f r, the radial momentum source is the inertial one (centrifugal
    and Coriolis terms are exactly the expansion of rho v_in^2 / r), and the
    azimuthal one is the inertial one less rho Omega_f u (along a parcel's
    path, d v / dt = d v_in / dt - Omega_f dr / dt).  A sign error in either
    Coriolis term or in the centrifugal term fails this."""
    from dataclasses import replace
    base = syn.scaled(syn.VORTEX, 12, 8, 16)
    rng = np.random.default_rng(12)
    for omega in (1.0, 0.63):
        o_rot = oracle.Oracle(replace(base, omega_frame=omega))
        o_in = oracle.Oracle(replace(base, omega_frame=0.0))
        rc, _ = o_rot.coords(0)
        for i, k in ((0, 0), (6, 9), (11, 15)):
            r = rc[i]
            U, (rho, u, v, ww, P, rd, ud, vd, wd) = _state(rng, base.gamma)
            Ui = U.copy()
            Ui[MV] = rho * (v + omega * r)
            Ui[EN] = P / (base.gamma - 1) + 0.5 * rho * (u * u + (v + omega * r) ** 2 + ww * ww)
            Ui[DMV] = rd * (vd + omega * r)
            Sr, Si = o_rot.sources(i, 1, k, U), o_in.sources(i, 1, k, Ui)
            scale = rho * (v + omega * r) ** 2 / r + P / r
            assert Sr[MU] == pytest.approx(Si[MU], abs=1e-12 * scale)
            assert Sr[MV] == pytest.approx(Si[MV] - rho * omega * u, abs=1e-12 * scale)
            assert Sr[DMU] == pytest.approx(Si[DMU], abs=1e-12 * scale)
            assert Sr[DMV] == pytest.approx(Si[DMV] - rd * omega * ud, abs=1e-12 * scale)
