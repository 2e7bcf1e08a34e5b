"""Epicyclic oscillation: a pin of the rotating-disc dynamics (the Coriolis,
centrifugal and geometric source terms, the rotating frame and the pressure
force together) against a closed form.

An axisymmetric radial velocity u_r = 1e-4 G(r) (a Gaussian of width 0.2 at
r0 = 1) on the stratified disc, in one periodic z cell (the midplane), in the
equal-Mach frame of the annulus r in [0.6, 1.6]: a fluid ring displaced
radially oscillates at the epicyclic frequency kappa, kappa^2 = (2 Omega / r)
d(r^2 Omega)/dr = Omega_K^2 for Keplerian rotation, raised by the pressure
term c_s^2 k^2 (~4 % for this width: kappa^2 + c_s^2 / 0.2^2).  The pin: the
period of u_r at r0 over one oscillation gives 0.97 <= omega / Omega_K(r0)
<= 1.06, and the amplitude does not grow, with the primitive-departure
option and with option 2 (the pressure departure in place of the energy
one).

With the paper's conservative-departure reconstruction the same run does
not oscillate: at this frame Mach number (~12 near r = 0.7) the component-
wise MinMod clips the momentum, energy and density departures at different
places, the face pressure (a difference of terms O(Mach^2) larger than
itself) takes spurious jumps, and u_r grows ~100-fold within one orbit near
r = 0.72.  Without the limiter, or with the primitive-departure option, it
oscillates as above.  That run is reported here, not pinned.

Where the instability sets in: on the narrow annulus r in [0.9, 1.1] with a
seed of width 0.03, the frame rate sets the largest frame Mach number of the
annulus.  Over one orbit the conservative reading keeps |u_r| at its seed up
to Mach 7.5 (Omega_f = 0.8) and grows it about 200-fold from Mach 9.6
(Omega_f = 0.7) on; the two options stay at their seed up to Mach 15.7
(Omega_f = 0.4).  Pinned at Mach 3.7, 7.5 and 11.6.
"""
from dataclasses import replace
import math

import numpy as np
import pytest

import oracle
import synthetic as syn

H = 0.05


def _run(recon, t_end):
    w = replace(syn.RWI, nr=128, nth=4, nz=1, x0=(0.6, 0.0, -0.5 * H), x1=(1.6, 2.0 * math.pi, 0.5 * H),
                rwi_delta=0.0, recon=recon,
                bc_lo=(syn.BC_EQUILIBRIUM, syn.BC_PERIODIC, syn.BC_PERIODIC),
                bc_hi=(syn.BC_EQUILIBRIUM, syn.BC_PERIODIC, syn.BC_PERIODIC))
    o = oracle.Oracle(w)
    E0 = o.equilibrium_state()
    r, _ = o.coords(0)
    u0 = 1e-4 * np.exp(-0.5 * ((r - 1.0) / 0.2) ** 2)
    E = E0.copy()
    E[0] = E0[4] * u0[None, None, :]
    E[3] = E0[3] + 0.5 * E0[4] * u0[None, None, :] ** 2
    i0 = int(np.argmin(np.abs(r - 1.0)))
    t, ts, us, umax = 0.0, [0.0], [u0[i0]], [u0.max()]
    while t < t_end:
        dt = o.cfl_dt(E)
        E = o.step(E, dt)
        if o.take_status():
            break
        t += dt
        u = E[0, 0, 0] / E[4, 0, 0]
        ts.append(t)
        us.append(u[i0])
        umax.append(np.abs(u).max())
    return np.array(ts), np.array(us), np.array(umax), u0.max()


@pytest.mark.parametrize("recon", [syn.RECON_PRIMITIVE, syn.RECON_PRESSURE], ids=["primitive", "pressure"])
def test_epicycle_frequency(recon):
    t, u, umax, a0 = _run(recon, 7.5)
    zc = t[1:][np.diff(np.sign(u)) != 0]  # zero crossings of u_r at r0
    assert len(zc) >= 2, zc
    omega = math.pi / (zc[1] - zc[0])     # half a period between consecutive crossings
    print(f"epicycle: omega / Omega_K(r0) = {omega:.4f}, max |u_r| over the run {umax.max():.3e} (seed {a0:.3e})")
    assert 0.97 <= omega <= 1.06, omega
    assert umax.max() <= 1.2 * a0


def test_epicycle_conservative_reconstruction_report():
    t, u, umax, a0 = _run(syn.RECON_CONSERVATIVE, 2.5)
    print("conservative reconstruction, max |u_r| / seed at t =",
          [(f"{t[k]:.2f}", f"{umax[k] / a0:.1f}") for k in range(0, len(t), max(1, len(t) // 8))])


def _narrow_growth(recon, omega_frame, t_end=6.3):
    """Largest |u_r| over one orbit on r in [0.9, 1.1], divided by the seed's."""
    w = replace(syn.RWI, nr=64, nth=4, nz=1, x0=(0.9, 0.0, -0.5 * H), x1=(1.1, 2.0 * math.pi, 0.5 * H),
                rwi_delta=0.0, recon=recon, omega_frame=omega_frame,
                bc_lo=(syn.BC_EQUILIBRIUM, syn.BC_PERIODIC, syn.BC_PERIODIC),
                bc_hi=(syn.BC_EQUILIBRIUM, syn.BC_PERIODIC, syn.BC_PERIODIC))
    o = oracle.Oracle(w)
    E0 = o.equilibrium_state()
    r, _ = o.coords(0)
    u0 = 1e-4 * np.exp(-0.5 * ((r - 1.0) / 0.03) ** 2)
    E = E0.copy()
    E[0] = E0[4] * u0[None, None, :]
    E[3] = E0[3] + 0.5 * E0[4] * u0[None, None, :] ** 2
    t, growth = 0.0, 1.0
    while t < t_end:
        dt = o.cfl_dt(E)
        E = o.step(E, dt)
        t += dt
        if o.take_status():
            return math.inf
        growth = max(growth, float(np.abs(E[0, 0, 0] / E[4, 0, 0]).max() / u0.max()))
    return growth


@pytest.mark.parametrize("omega_frame,stable", [(1.0, True), (0.8, True), (0.6, False)],
                         ids=["mach_3.7", "mach_7.5", "mach_11.6"])
def test_conservative_reading_stability_threshold(omega_frame, stable):
    g_cons = _narrow_growth(syn.RECON_CONSERVATIVE, omega_frame)
    g_pres = _narrow_growth(syn.RECON_PRESSURE, omega_frame)
    print(f"Omega_f = {omega_frame}: max |u_r| / seed, conservative {g_cons:.2f}, option 2 {g_pres:.2f}")
    assert g_pres <= 1.2
    if stable:
        assert g_cons <= 1.2
    else:
        assert g_cons >= 10.0


@pytest.mark.parametrize("omega_frame", [0.0, 0.8036, 1.0], ids=["inertial", "equal_mach", "co_rotating"])
def test_dust_epicycle_frequency(omega_frame):
    """A pressureless dust ring (1 % of the gas density, Keplerian, drag
    negligible: St = 1e12) given u_r = 1e-4 exp(-(r - 1)^2 / (2 0.1^2)): each
    ring of test particles oscillates at kappa = Omega_K exactly, whatever
    the frame.  Pins the dust's geometric, gravity, centrifugal and Coriolis
    terms in the rotating frame (measured 0.9979, 1.0010, 1.0018 over two
    orbits at 64 radial cells, amplitude kept to 1 %)."""
    w = replace(syn.RWI, nr=64, nth=4, nz=1, x0=(0.6, 0.0, -0.5 * H), x1=(1.6, 2.0 * math.pi, 0.5 * H),
                rwi_delta=0.0, omega_frame=omega_frame, n_dust=1, stokes=1e12, drag_law=0,
                bc_lo=(syn.BC_EQUILIBRIUM, syn.BC_PERIODIC, syn.BC_PERIODIC),
                bc_hi=(syn.BC_EQUILIBRIUM, syn.BC_PERIODIC, syn.BC_PERIODIC))
    o = oracle.Oracle(w)
    E = o.equilibrium_state()
    r, _ = o.coords(0)
    rd = 0.01 * E[4]
    u0 = 1e-4 * np.exp(-0.5 * ((r - 1.0) / 0.1) ** 2)[None, None, :]
    E[8] = rd
    E[5] = rd * u0
    E[6] = rd * (np.sqrt(w.gm / r) - omega_frame * r)[None, None, :]
    i0 = int(np.argmin(np.abs(r - 1.0)))
    t, ts, us = 0.0, [0.0], [u0[0, 0, i0]]
    while t < 4.0 * math.pi:
        dt = o.cfl_dt(E)
        E = o.step(E, dt)
        t += dt
        ts.append(t)
        us.append(E[5, 0, 0, i0] / E[8, 0, 0, i0])
    assert o.take_status() == 0
    ts, us = np.array(ts), np.array(us)
    k = np.nonzero(np.sign(us[1:]) != np.sign(us[:-1]))[0]
    zc = ts[k] - us[k] * (ts[k + 1] - ts[k]) / (us[k + 1] - us[k])   # interpolated zero crossings
    omega = math.pi / np.mean(np.diff(zc))
    print(f"dust epicycle, Omega_f = {omega_frame}: omega / Omega_K(r0) = {omega:.5f} ({len(zc)} crossings)")
    assert len(zc) >= 3
    assert abs(omega - 1.0) <= 0.01
    assert np.abs(us).max() <= 1.01 * u0.max()
