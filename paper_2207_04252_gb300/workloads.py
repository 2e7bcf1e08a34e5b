"""Grids and initial states of the synthetic workloads, on the CUDA side.

``Grid`` wraps a library grid built from a ``synthetic.Workload``.  The
initial-condition recipes are written here from the workload descriptions
(this side's own restatement; the CPU oracle has its own).  Only the seeded
noise comes from the shared ``synthetic`` package.

Recipes (all on the library's equilibrium E0):
  sod    : (rho, p, u) = (1, 1, 0) for x < 0.5, (0.125, 0.1, 0) otherwise.
  noise  : rho' = a xi rho0 at fixed velocity and pressure, so
           (rho v)' = rho' v0 and E' = rho' v0^2 / 2.
  vortex : Gaussian stream function psi = psi0 exp(-(r-rv)^2/(2 s_r^2)
           - (rv dtheta)^2/(2 s_t^2)), s_r = width * H(rv), s_t = chi s_r,
           psi0 set by the centre vorticity -amp * (3/2) Omega_K(rv);
           u' = (1/r) dpsi/dtheta, v' = -dpsi/dr, rho and P at equilibrium.
           Dust: rho_d = ratio rho0 (1 + a_d xi_d), moving with the gas; with
           several species each takes ratio / n of it, with its own noise.
  rwi    : the equilibrium carries the radial density bump (rho, P x (1 +
           delta G), G a Gaussian at r0, v_theta0 in radial balance with it:
           rossbi_disc_params' bump); the departure is the seed
           v_r = eps v_theta0 sin(m theta) G (v_theta0 inertial).
"""
import math

import numpy as np
import torch

import synthetic as syn

from . import rossbi as R


class Grid:
    def __init__(self, w: syn.Workload, precision: int = R.ROSSBI_FP64, stream=None):
        self.w = w
        self.precision = precision
        desc = R.make_desc(w.geometry, (w.nr, w.nth, w.nz), w.x0, w.x1, w.bc_lo, w.bc_hi, w.gamma, w.gm,
                           w.omega_frame, w.cfl, w.n_dust, precision, w.recon)
        self.h = R.rossbi_init_grid(desc, stream)
        try:
            R.rossbi_set_equilibrium(self.h, w.disc_params())
        except Exception:
            R.rossbi_destroy(self.h)
            self.h = None
            raise
        self.nf = R.rossbi_nfields(self.h)
        self.dtype = torch.float32 if precision == R.ROSSBI_FP32_PERT else torch.float64
        self.perturbation = precision in (R.ROSSBI_FP32_PERT, R.ROSSBI_FP64_PERT)
        self.dust = (w.stokes, w.drag_law, w.drag_kappa) if w.n_dust else None
        self.shape = (self.nf, w.nz, w.nth, w.nr)
        if w.dust_stokes_factors:
            R.rossbi_set_dust_species(self.h, w.dust_stokes_factors)

    def close(self):
        if self.h:
            R.rossbi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- library calls
    def step(self, state, dt=0.0, scratch=None, want_next_dt=False):
        return R.rossbi_step(self.h, state, scratch, dt, self.dust, want_next_dt)

    def adjoint_step(self, state, dt, lam_np1, lam_n=None, want_dstokes=False):
        """Cotangent of E^n from that of E^{n+1} (in place when lam_n is None)."""
        return R.rossbi_adjoint_step(self.h, state, dt, self.dust, lam_np1, lam_np1 if lam_n is None else lam_n,
                                     want_dstokes)

    def cfl_dt(self, state):
        return R.rossbi_cfl_dt(self.h, state)

    def set_indirect(self, x_ref):
        """Indirect gravity of Sect. 2.10 with constant X_ref (0 = off)."""
        R.rossbi_set_indirect(self.h, x_ref)

    def set_damping(self, zones):
        """Wave-killing zones (r_edge_in, r_edge_out, period_factor), or None."""
        R.rossbi_set_damping(self.h, zones)

    def set_vertical_damping(self, zone):
        """Vertical sheared damped boundary (z_edge, period_factor), or None."""
        R.rossbi_set_vertical_damping(self.h, zone)

    def indirect_moments(self, state):
        """(A_disc, B_disc) of Sect. 2.10 of a state, FP64."""
        return R.rossbi_indirect_moments(self.h, state)

    def sums(self, state):
        return R.rossbi_conservation_sums(self.h, state)

    def take_status(self):
        return R.rossbi_take_status(self.h)

    def equilibrium(self) -> np.ndarray:
        """E0 at cell centres, (5, nz, nr), float64."""
        return R.rossbi_get_equilibrium(self.h, self.w.nz, self.w.nr)

    # ---- mesh (Sect. 2.3), restated for building inputs
    def centres(self, ax):
        w = self.w
        n = (w.nr, w.nth, w.nz)[ax]
        if ax == 0 and w.geometry == syn.GEOM_CYL:
            f = w.x0[0] * (w.x1[0] / w.x0[0]) ** (np.arange(n + 1) / n)
            return np.sqrt(f[:-1] * f[1:])
        return w.x0[ax] + (np.arange(n) + 0.5) * (w.x1[ax] - w.x0[ax]) / n

    # ---- inputs
    def _vortex_velocity(self, amp):
        """Velocity perturbation (u', v') of the vortex recipe, (1, nth, nr) each; linear in amp."""
        w = self.w
        r = self.centres(0)[None, None, :]
        th = self.centres(1)[None, :, None]
        sigma0, beta_sigma, T0, beta_T = w.disc
        up = np.zeros((1, w.nth, w.nr))
        vp = np.zeros((1, w.nth, w.nr))
        for rv, thv in w.vortices:
            omk = math.sqrt(w.gm / rv ** 3)
            s_r = w.vortex_width_h * math.sqrt(2.0 * T0 * rv ** beta_T) / omk
            s_t = w.vortex_chi * s_r
            psi0 = -amp * 1.5 * omk / (1.0 / s_r ** 2 + 1.0 / s_t ** 2)
            dth = np.mod(th - thv + math.pi, 2.0 * math.pi) - math.pi
            psi = psi0 * np.exp(-(r - rv) ** 2 / (2.0 * s_r ** 2) - (rv * dth) ** 2 / (2.0 * s_t ** 2))
            up = up - psi * rv * rv * dth / (r * s_t ** 2)
            vp = vp + psi * (r - rv) / s_r ** 2
        return up, vp

    def vortex_amp_tangent(self) -> np.ndarray:
        """dE/d(vortex amplitude) of the initial state, (nf, nz, nth, nr), float64."""
        w = self.w
        assert w.ic == "vortex"
        E0 = self.equilibrium()
        rho0 = E0[syn.F_RHO][:, None, :]
        v0 = (E0[syn.F_MV] / E0[syn.F_RHO])[:, None, :]
        up, vp = self._vortex_velocity(w.vortex_amp)
        u1, v1 = self._vortex_velocity(1.0)
        T = np.zeros(self.shape)
        T[syn.F_MU] = rho0 * u1
        T[syn.F_MV] = rho0 * v1
        T[syn.F_EN] = rho0 * (up * u1 + v0 * v1 + vp * v1)
        for b, rd in self._dust_densities(rho0):
            T[b] = rd * u1
            T[b + 1] = rd * v1
        return T

    def _dust_densities(self, rho0):
        """(first field, initial density) of each dust species: an equal share
        of the dust-to-gas ratio, with the species' own seeded noise."""
        w = self.w
        nd = (self.nf - 5) // 4
        out = []
        for s in range(nd):
            xi = syn.uniform_pm1(w.seed, syn.F_DRHO + 4 * s, w.ncell).reshape(w.nz, w.nth, w.nr)
            out.append((5 + 4 * s, w.dust_ratio / nd * rho0 * (1.0 + w.dust_noise * xi)))
        return out

    def dust_velocity(self) -> np.ndarray:
        """Initial dust velocity (u, v, w), (3, nz, nth, nr): the gas velocity of the recipe."""
        w = self.w
        E0 = self.equilibrium()
        v0 = (E0[syn.F_MV] / E0[syn.F_RHO])[:, None, :]
        up, vp = self._vortex_velocity(w.vortex_amp) if w.ic == "vortex" else (0.0, 0.0)
        out = np.zeros((3, w.nz, w.nth, w.nr))
        out[0] = up
        out[1] = v0 + vp
        return out

    def perturbation_state(self) -> np.ndarray:
        """E - E0 in float64, (nf, nz, nth, nr), for the workload's recipe."""
        w = self.w
        g = w.gamma
        Ep = np.zeros(self.shape)
        if w.ic == "sod":
            left = self.centres(0) < 0.5
            Ep[syn.F_RHO] = np.where(left, 1.0, 0.125)[None, None, :]
            Ep[syn.F_EN] = (np.where(left, 1.0, 0.1) / (g - 1.0))[None, None, :]
            return Ep
        if w.ic == "explosion":  # at rest; (rho, P) = (1, 1) inside r = 0.4, (0.125, 0.1) outside
            high = self.centres(0) <= 0.4
            Ep[syn.F_RHO] = np.where(high, 1.0, 0.125)[None, None, :]
            Ep[syn.F_EN] = (np.where(high, 1.0, 0.1) / (g - 1.0))[None, None, :]
            return Ep
        E0 = self.equilibrium()
        rho0 = E0[syn.F_RHO][:, None, :]
        v0 = (E0[syn.F_MV] / E0[syn.F_RHO])[:, None, :]
        if w.ic == "noise":
            xi = syn.uniform_pm1(w.seed, syn.F_RHO, w.ncell).reshape(w.nz, w.nth, w.nr)
            drho = w.noise_amp * xi * rho0
            Ep[syn.F_RHO] = drho
            Ep[syn.F_MV] = drho * v0
            Ep[syn.F_EN] = 0.5 * drho * v0 * v0
            return Ep
        if w.ic == "rwi":  # the density bump belongs to the equilibrium; only the seeded v_r of mode m departs
            r = self.centres(0)[None, None, :]
            th = self.centres(1)[None, :, None]
            G = np.exp(-((r - w.rwi_r0) / (math.sqrt(2.0) * w.rwi_width)) ** 2)
            vth0 = v0 + w.omega_frame * r  # the inertial equilibrium azimuthal velocity
            vr = w.rwi_eps * vth0 * np.sin(w.rwi_mode * th) * G
            Ep[syn.F_MU] = rho0 * vr
            Ep[syn.F_EN] = 0.5 * rho0 * vr * vr
            return Ep
        if w.ic != "vortex":
            raise ValueError(w.ic)
        up, vp = self._vortex_velocity(w.vortex_amp)
        Ep[syn.F_MU] = rho0 * up
        Ep[syn.F_MV] = rho0 * vp
        Ep[syn.F_EN] = 0.5 * rho0 * (up * up + 2.0 * v0 * vp + vp * vp)
        for b, rd in self._dust_densities(rho0):
            Ep[b + 3] = rd
            Ep[b] = rd * up
            Ep[b + 1] = rd * (v0 + vp)
        return Ep

    def initial_state(self, device="cuda") -> torch.Tensor:
        """Initial state in this grid's precision form, on `device`."""
        Ep = self.perturbation_state()
        if not self.perturbation:
            Ep[:5] += self.equilibrium()[:, :, None, :]
        return torch.from_numpy(Ep).to(device=device, dtype=self.dtype).contiguous()

    def full_state(self, state) -> np.ndarray:
        """Full conservative E in float64 on the host (E0 + E' for the perturbation forms)."""
        E = state.detach().to("cpu", torch.float64).numpy().copy()
        if self.perturbation:
            E[:5] += self.equilibrium()[:, :, None, :]
        return E
