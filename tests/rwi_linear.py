"""Linear growth rates of the Rossby wave instability (Sect. 4.3) of the
bumped disc, for the tests.

The paper measures the RWI by the growth rates of the azimuthal modes m and
compares them with those of a cited work.  This module gives the rates the
discrete runs are held to: the eigenvalues of the linearised 2-D equations of
an inviscid, adiabatic gas (ratio of specific heats gamma) orbiting a point
mass, about an axisymmetric equilibrium rho_0(r), P_0(r), Omega(r) in radial
balance, for perturbations proportional to exp(i (m theta - omega t)):

    -i w' rho' + (1/r) d(r rho_0 u)/dr + i m rho_0 v / r = 0
    -i w' u - 2 Omega v = -(1/rho_0) dP'/dr + rho' P_0' / rho_0^2
    -i w' v + (kappa^2 / 2 Omega) u = -i m P' / (rho_0 r)
    -i w' P' + u P_0' + gamma P_0 ((1/r) d(r u)/dr + i m v / r) = 0

with w' = omega - m Omega(r) and kappa^2 = (2 Omega / r) d(r^2 Omega)/dr
(u, v the radial and azimuthal velocity perturbations).  They are discretised
by second-order differences on a uniform radial mesh, u on the faces (zero on
the two end faces: reflecting walls), rho', v and P' at the centres, and the
dense eigenproblem omega X = M X is solved.  An unstable RWI mode is an
eigenvalue with Im(omega) > 0 and its corotation Re(omega) / m = Omega(r) at
the bump.  The equilibrium is passed in as a function of r; the tests take
the oracle's midplane equilibrium (its radial and vertical balance are pinned
on their own).  This is test infrastructure: no product code calls it.
"""
import numpy as np
import scipy.linalg as sl


def rwi_modes(background, m, r_in, r_out, n=400, gamma=1.4):
    """All eigenvalues omega of mode m on r in [r_in, r_out] with n cells,
    sorted by decreasing Im(omega).

    background(r) -> (rho_0, v_theta_0, P_0) at radius r (inertial frame)."""
    rf = np.linspace(r_in, r_out, n + 1)
    rc = 0.5 * (rf[1:] + rf[:-1])
    dr = rf[1] - rf[0]

    def bg(r):
        a = np.array([background(x) for x in np.atleast_1d(r)])
        return a[:, 0], a[:, 1] / np.atleast_1d(r), a[:, 2]

    h = 1e-5 * (r_out - r_in)

    def dpdr(r):
        return (bg(r + h)[2] - bg(r - h)[2]) / (2.0 * h)

    def kappa2(r):
        def L(x):
            return x * x * bg(x)[1]
        return 2.0 * bg(r)[1] / r * (L(r + h) - L(r - h)) / (2.0 * h)

    rho_c, om_c, p_c = bg(rc)
    rho_f, om_f, _ = bg(rf)
    dp_c, dp_f = dpdr(rc), dpdr(rf)
    k2_c = kappa2(rc)

    nu = n - 1                      # interior faces 1 .. n-1
    rfi = rf[1:-1]
    # centre <- face: average and difference (u = 0 on the end faces)
    a_fc = np.zeros((n, nu))
    d_fc = np.zeros((n, nu))
    for i in range(n):
        for jf, s in ((i, -1.0), (i + 1, 1.0)):
            if 1 <= jf <= n - 1:
                a_fc[i, jf - 1] += 0.5
                d_fc[i, jf - 1] += s / dr
    # face <- centre: average and difference
    a_cf = np.zeros((nu, n))
    d_cf = np.zeros((nu, n))
    for j in range(1, n):
        a_cf[j - 1, j - 1] = a_cf[j - 1, j] = 0.5
        d_cf[j - 1, j - 1], d_cf[j - 1, j] = -1.0 / dr, 1.0 / dr

    iR, iU, iV, iP = 0, n, n + nu, 2 * n + nu
    M = np.zeros((3 * n + nu, 3 * n + nu), complex)
    # omega X = m Omega X + i (rest of each equation solved for d/dt)
    M[iR:iR + n, iR:iR + n] += np.diag(m * om_c)
    M[iR:iR + n, iU:iU + nu] += -1j * d_fc * (rfi * rho_f[1:-1])[None, :] / rc[:, None]
    M[iR:iR + n, iV:iV + n] += np.diag(m * rho_c / rc)
    M[iU:iU + nu, iU:iU + nu] += np.diag(m * om_f[1:-1])
    M[iU:iU + nu, iV:iV + n] += 2j * om_f[1:-1, None] * a_cf
    M[iU:iU + nu, iP:iP + n] += -1j * d_cf / rho_f[1:-1, None]
    M[iU:iU + nu, iR:iR + n] += 1j * a_cf * (dp_f[1:-1] / rho_f[1:-1] ** 2)[:, None]
    M[iV:iV + n, iV:iV + n] += np.diag(m * om_c)
    M[iV:iV + n, iU:iU + nu] += -1j * (k2_c / (2.0 * om_c))[:, None] * a_fc
    M[iV:iV + n, iP:iP + n] += np.diag(m / (rho_c * rc))
    M[iP:iP + n, iP:iP + n] += np.diag(m * om_c)
    M[iP:iP + n, iU:iU + nu] += -1j * (dp_c[:, None] * a_fc + gamma * p_c[:, None] * d_fc * rfi[None, :] / rc[:, None])
    M[iP:iP + n, iV:iV + n] += np.diag(gamma * p_c * m / rc)
    ev = sl.eigvals(M)
    return ev[np.argsort(-ev.imag)]


def rwi_growth_rate(background, m, r0, r_in, r_out, n=400, gamma=1.4, window=0.1):
    """Largest Im(omega) among the modes whose corotation radius is the bump's:
    |Re(omega) / (m Omega(r0)) - 1| < window.  0 when there is none."""
    ev = rwi_modes(background, m, r_in, r_out, n, gamma)
    om0 = background(r0)[1] / r0
    near = [e.imag for e in ev if abs(e.real / (m * om0) - 1.0) < window]
    return max(max(near, default=0.0), 0.0)
