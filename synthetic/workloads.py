"""Workload descriptions: the synthetic stand-ins for the paper's test problems.

The paper's own workloads (Sect. 4: cylindrical explosion, equilibrium disc,
Rossby-wave vortices, dust trapping; the "column Gaussian vortex" of its
scaling runs) use no public dataset.  These six describe the sizes, extents,
parameters and seeds of the synthetic inputs; the initial-condition recipe is
written out independently by each side.

Disc parameters: aspect ratio h = H/r = 0.05 with T ~ r^-1, so the locally
isothermal temperature normalisation is T0 = h^2/2; Sigma ~ r^-0.5; gamma = 1.4;
GM = 1.  The vertical extent is +-3 H(r=1) = +-0.15 and r spans [0.5, 2] on a
logarithmic mesh.

Frame rotation (the paper does not give it).  The vortex workloads co-rotate
with the vortex at r = 1 (Omega_f = Omega_K(1) = 1).  The bare noisy disc uses
the rate that makes the frame-relative Mach number equal, and so smallest, at
the two radial edges: with v_K = r^-1/2 and c ~ r^-1/2 that is
Omega_f = 2 / (r_in^1.5 + r_out^1.5) (Mach ~19 at both edges instead of 44
at r = 2 for Omega_f = 1).
"""
from dataclasses import dataclass, field, replace
import math

GEOM_BOX, GEOM_CYL = 0, 1
BC_PERIODIC, BC_OUTFLOW, BC_EQUILIBRIUM = 0, 1, 2
F_MU, F_MV, F_MW, F_EN, F_RHO, F_DMU, F_DMV, F_DMW, F_DRHO = range(9)
# Gas reconstruction: the paper's component-wise parabola on the conservative
# departures (Sect. 2.7 on App. B's E), or the primitive-departure option.
RECON_CONSERVATIVE, RECON_PRIMITIVE, RECON_PRESSURE = 0, 1, 2

H_ASPECT = 0.05
DISC_PARAMS = (1.0, -0.5, H_ASPECT * H_ASPECT / 2.0, -1.0)  # sigma0, beta_sigma, T0, beta_T
Z_HALF = 3.0 * H_ASPECT


@dataclass(frozen=True)
class Workload:
    name: str
    geometry: int
    nr: int
    nth: int
    nz: int
    x0: tuple
    x1: tuple
    bc_lo: tuple
    bc_hi: tuple
    ic: str                      # "sod", "noise", "vortex", "explosion", "rwi"
    steps: int
    gamma: float = 1.4
    gm: float = 1.0
    omega_frame: float = 1.0
    cfl: float = 0.5
    n_dust: int = 0
    disc: tuple = None           # (sigma0, beta_sigma, T0, beta_T) or None; see disc_params
    seed: int = 0
    noise_amp: float = 0.0       # relative gas-density noise amplitude
    vortices: tuple = ()         # ((r_v, theta_v), ...)
    vortex_amp: float = 0.2      # centre vorticity / local shear rate (3/2 Omega_K)
    vortex_chi: float = 4.0      # azimuthal / radial Gaussian width
    vortex_width_h: float = 2.0  # radial width in units of H(r_v)
    dust_ratio: float = 0.0
    dust_noise: float = 0.0
    stokes: float = 0.0
    drag_law: int = 0
    drag_kappa: float = 0.0      # drag law 2: r_p / lambda_0 of the Stokes regime
    t_end: float = 0.0           # >0: run to this time, clipping the last step
    checkpoint_every: int = 0
    recon: int = RECON_CONSERVATIVE
    dust_stokes_factors: tuple = ()  # several species: St of species s = stokes x factor[s] (factor[0] = 1)
    rwi_mode: int = 0            # "rwi": azimuthal mode m of the seed
    rwi_delta: float = 0.0       # relative amplitude of the equilibrium's density bump
    rwi_width: float = 0.0       # Delta_r of the bump
    rwi_eps: float = 0.0         # seed amplitude, v_r = eps v_theta0 sin(m theta) G(r)
    rwi_r0: float = 1.0          # radius of the bump

    def disc_params(self):
        """The equilibrium's seven parameters (sigma0, beta_sigma, T0, beta_T,
        bump_delta, bump_r0, bump_width) as both libraries take them: the
        radial density bump only on the "rwi" workloads, else delta = 0."""
        if self.disc is None:
            return None
        bump = (self.rwi_delta, self.rwi_r0, self.rwi_width) if self.ic == "rwi" else (0.0, 1.0, 0.0)
        return tuple(self.disc) + bump

    @property
    def ncell(self) -> int:
        return self.nr * self.nth * self.nz

    @property
    def nfields(self) -> int:
        return 5 + 4 * self.n_dust

    @property
    def shape(self) -> tuple:
        return (self.nfields, self.nz, self.nth, self.nr)


def equal_mach_frame(r_in: float, r_out: float) -> float:
    """Frame angular speed with equal frame Mach numbers at both radial edges (GM = 1, T ~ 1/r)."""
    return 2.0 / (r_in ** 1.5 + r_out ** 1.5)


def _disc(name, nr, nth, nz, steps, **kw) -> Workload:
    return Workload(
        name=name, geometry=GEOM_CYL, nr=nr, nth=nth, nz=nz,
        x0=(0.5, 0.0, -Z_HALF), x1=(2.0, 2.0 * math.pi, Z_HALF),
        bc_lo=(BC_EQUILIBRIUM, BC_PERIODIC, BC_EQUILIBRIUM),
        bc_hi=(BC_EQUILIBRIUM, BC_PERIODIC, BC_EQUILIBRIUM),
        disc=DISC_PARAMS, steps=steps, **kw)


# Sod shock tube along x in a 256x4x4 Box (gamma = 1.4, diaphragm at x = 0.5, t = 0.2).
SOD = Workload(
    name="sod_box_256x4x4", geometry=GEOM_BOX, nr=256, nth=4, nz=4,
    x0=(0.0, 0.0, 0.0), x1=(1.0, 4.0 / 256, 4.0 / 256),
    bc_lo=(BC_OUTFLOW, BC_PERIODIC, BC_PERIODIC), bc_hi=(BC_OUTFLOW, BC_PERIODIC, BC_PERIODIC),
    ic="sod", steps=0, omega_frame=0.0, t_end=0.2)

# Stratified Keplerian disc equilibrium with 1e-4 seeded density noise, gas only.
DISC_NOISE = _disc("disc_eq_noise_128x256x32", 128, 256, 32, 100, ic="noise", seed=2207, noise_amp=1e-4,
                   omega_frame=equal_mach_frame(0.5, 2.0))

# Bi-fluid disc with one Gaussian vortex at r = 1, St = 0.1, dust/gas = 0.01 (+1e-3 noise).
VORTEX = _disc("bifluid_vortex_256x512x64", 256, 512, 64, 200, ic="vortex", n_dust=1, seed=4252,
               vortices=((1.0, math.pi),), dust_ratio=0.01, dust_noise=1e-3, stokes=0.1)

# Adjoint workload: the bi-fluid vortex at 128x256x32, checkpoints every 20 steps.
ADJOINT = _disc("adjoint_vortex_128x256x32", 128, 256, 32, 200, ic="vortex", n_dust=1, seed=2207,
                vortices=((1.0, math.pi),), dust_ratio=0.01, dust_noise=1e-3, stokes=0.1,
                checkpoint_every=20)

# Throughput workload: 512x1024x128 (~67M cells), two vortices, St = 0.05.
THROUGHPUT = _disc("bifluid_two_vortices_512x1024x128", 512, 1024, 128, 50, ic="vortex", n_dust=1,
                   seed=4252, vortices=((0.8, 0.0), (1.3, math.pi)), dust_ratio=0.01, dust_noise=1e-3,
                   stokes=0.05)

# Rossby wave instability (Sect. 4.3): a radial Gaussian density bump in the
# stationary solution, rho = rho0 (1 + delta G), G = exp(-((r - r0)/(sqrt(2)
# Delta_r))^2), at the equilibrium temperature (P scaled alike) with the
# azimuthal velocity in radial balance with the bump's pressure gradient, and
# the seed v_r = eps v_theta0 sin(m theta) G with eps = 1e-4 and mode m.  The
# paper takes the setup of a cited work without printing delta and Delta_r.
# In this disc (h = 0.05, T ~ 1/r, adiabatic perturbations with gamma = 7/5)
# the linearised equations give no mode growing faster than 1e-3 Omega(r0)
# for a bump as wide as H(r0) = 0.05 (delta up to 3); delta = 0.5 and
# Delta_r = 0.025 r0 (= H(r0) / 2) give growth rates 0.06 to 0.14 Omega(r0)
# for m = 2 ... 6 (0.111 for m = 4) and keep kappa^2 > 0.33 Omega^2
# (delta = 1 at this width is Rayleigh-marginal).  The annulus r in
# [0.6, 1.6] has 256 log-spaced cells (6.5 per Delta_r); z in +-2 H(r0);
# gas only, in the annulus's equal-Mach frame.
RWI = Workload(
    name="rwi_m4_256x256x16", geometry=GEOM_CYL, nr=256, nth=256, nz=16,
    x0=(0.6, 0.0, -2.0 * H_ASPECT), x1=(1.6, 2.0 * math.pi, 2.0 * H_ASPECT),
    bc_lo=(BC_EQUILIBRIUM, BC_PERIODIC, BC_EQUILIBRIUM), bc_hi=(BC_EQUILIBRIUM, BC_PERIODIC, BC_EQUILIBRIUM),
    disc=DISC_PARAMS, ic="rwi", steps=4000, rwi_mode=4, rwi_delta=0.5, rwi_width=0.025, rwi_eps=1e-4,
    omega_frame=equal_mach_frame(0.6, 1.6))

# Cylindrical explosion (Sect. 4.1; Toro ch. 17): a 2-D Riemann problem on the
# polar mesh, (rho, P) = (1, 1) for r <= 0.4 and (0.125, 0.1) outside, at rest;
# no gravity, no rotation, no equilibrium, gamma = 1.4; N_r x N_theta =
# 1600 x 3200 with one z cell.  The paper gives no radial extent: r in
# [e^-pi, 1] makes every cell of the logarithmic mesh square at this
# resolution (dr / r = dtheta).  The single z cell is thick (dz = 1) so that
# the CFL step is set by the r and theta faces.  Run to t = 0.25, the time of
# Toro's reference solution (the paper prints t = 2.5).
EXPLOSION = Workload(
    name="explosion_polar_1600x3200x1", geometry=GEOM_CYL, nr=1600, nth=3200, nz=1,
    x0=(math.exp(-math.pi), 0.0, -0.5), x1=(1.0, 2.0 * math.pi, 0.5),
    bc_lo=(BC_OUTFLOW, BC_PERIODIC, BC_PERIODIC), bc_hi=(BC_OUTFLOW, BC_PERIODIC, BC_PERIODIC),
    ic="explosion", steps=0, gm=0.0, omega_frame=0.0, t_end=0.25)

ALL = (SOD, DISC_NOISE, VORTEX, ADJOINT, THROUGHPUT, EXPLOSION, RWI)


def by_name(name: str) -> Workload:
    for w in ALL:
        if w.name == name:
            return w
    raise KeyError(name)


def scaled(w: Workload, nr: int, nth: int, nz: int, steps: int = None, **kw) -> Workload:
    """Same workload on another grid (same extents and physics); for tests."""
    x1 = w.x1
    if w.geometry == GEOM_BOX and w.ic == "sod":
        x1 = (w.x1[0], nth * (w.x1[0] - w.x0[0]) / nr, nz * (w.x1[0] - w.x0[0]) / nr)
    return replace(w, name=f"{w.name}@{nr}x{nth}x{nz}", nr=nr, nth=nth, nz=nz, x1=x1,
                   steps=w.steps if steps is None else steps, **kw)
