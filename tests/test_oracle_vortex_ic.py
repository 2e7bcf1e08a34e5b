"""The vortex initial condition of the bi-fluid workloads (reading R14) against
its definition.

The recipe adds to the disc the velocity field of a Gaussian stream function
psi (radial width 2 H(r_v), azimuthal width chi times that), u' = (1/r)
dpsi/dtheta, v' = -dpsi/dr, scaled so that the vortex's relative vorticity at
its centre is omega_c = -amp (3/2) Omega_K(r_v), an anticyclone of amplitude
amp in units of the Keplerian shear rate.  Independent of the closed forms
the oracle evaluates, central differences of the oracle's own initial
velocities must give: zero divergence, (1/r) d(r u')/dr + (1/r) dv'/dtheta
(a field derived from a stream function carries no compression), and a
vorticity (1/r) d(r v')/dr - (1/r) du'/dtheta equal to omega_c at the
centre; the dust moves with the gas.  A sign error, a missing 1/r or a
swapped width in either velocity component fails one of them.
"""
from dataclasses import replace
import math

import numpy as np

import oracle
import synthetic as syn


def test_vortex_velocity_is_solenoidal_with_the_prescribed_vorticity():
    # a fine grid on the vortex: r log-symmetric about r_v = 1 and theta
    # symmetric about theta_v = pi, odd counts so that a cell centre is the
    # vortex centre
    w = replace(syn.VORTEX, nr=201, nth=201, nz=1, x0=(0.8, math.pi - 0.5, -0.005),
                x1=(1.25, math.pi + 0.5, 0.005), vortices=((1.0, math.pi),), dust_noise=0.0)
    o = oracle.Oracle(w)
    E = oracle.initial_state(o)
    E0 = o.equilibrium_state()
    r, _ = o.coords(0)
    th, _ = o.coords(1)
    i0, j0 = w.nr // 2, w.nth // 2
    assert abs(r[i0] - 1.0) < 1e-12 and abs(th[j0] - math.pi) < 1e-12
    rho = E[syn.F_RHO, 0]
    u = E[syn.F_MU, 0] / rho
    v = E[syn.F_MV, 0] / rho - E0[syn.F_MV, 0] / E0[syn.F_RHO, 0]
    R = r[None, :]
    # central differences on the interior (theta uniform, r log-spaced)
    dth = th[1] - th[0]

    def d_r(f):
        return (f[:, 2:] - f[:, :-2]) / (R[:, 2:] - R[:, :-2])

    def d_th(f):
        return (f[2:, :] - f[:-2, :]) / (2.0 * dth)

    Ri = R[:, 1:-1]
    div = d_r(R * u)[1:-1, :] / Ri + d_th(v)[:, 1:-1] / Ri
    vort = d_r(R * v)[1:-1, :] / Ri - d_th(u)[:, 1:-1] / Ri
    omega_c = -w.vortex_amp * 1.5 * math.sqrt(w.gm / 1.0 ** 3)
    print(f"vorticity at the centre {vort[j0 - 1, i0 - 1]:.6f} (omega_c {omega_c}), max |div| {np.abs(div).max():.2e}")
    assert abs(vort[j0 - 1, i0 - 1] / omega_c - 1.0) < 1e-3
    assert np.abs(div).max() < 1e-3 * abs(omega_c)
    # along theta the vorticity is extremal at the centre (along r the
    # cylindrical terms move the extremum by about one cell), and
    # the velocity vanishes there
    assert np.argmin(vort[:, i0 - 1]) == j0 - 1
    assert abs(u[j0, i0]) < 1e-15 and abs(v[j0, i0]) < 1e-15
    # the dust moves with the gas
    rd = E[syn.F_DRHO, 0]
    np.testing.assert_allclose(E[syn.F_DMU, 0] / rd, u, rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(E[syn.F_DMV, 0] / rd, E[syn.F_MV, 0] / rho, rtol=1e-13, atol=1e-16)
