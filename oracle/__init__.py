"""TEST INFRASTRUCTURE ONLY: Python access to the FP64 CPU oracle.

The oracle (``rossbi_oracle.cpp``) is a plain, slow restatement of one
RoSSBi3D time step written from the paper.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import this
package.  It imports nothing from the CUDA package; the two share only the
seeded inputs of ``synthetic``.

The initial-condition recipes below are this side's own restatement of the
workload descriptions in ``synthetic.workloads``.
"""
import ctypes
import math
import os
import subprocess

import numpy as np

import synthetic as syn

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rossbi_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "librossbi_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with the host C++ compiler (FP contraction off)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = f"{_LIB}.{os.getpid()}.tmp"
    subprocess.check_call(["g++", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c++17",
                           "-o", tmp, _SRC])
    os.replace(tmp, _LIB)
    return _LIB


class _Desc(ctypes.Structure):
    _fields_ = [("geometry", ctypes.c_int), ("nr", ctypes.c_int), ("nth", ctypes.c_int), ("nz", ctypes.c_int),
                ("x0", ctypes.c_double * 3), ("x1", ctypes.c_double * 3),
                ("bc_lo", ctypes.c_int * 3), ("bc_hi", ctypes.c_int * 3),
                ("gamma", ctypes.c_double), ("gm", ctypes.c_double), ("omega_frame", ctypes.c_double),
                ("cfl", ctypes.c_double), ("n_dust", ctypes.c_int)]


_D = ctypes.POINTER(ctypes.c_double)
_L = ctypes.POINTER(ctypes.c_long)


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [ctypes.POINTER(_Desc)]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_nfields.argtypes = [ctypes.c_void_p]
        L.orc_set_equilibrium.argtypes = [ctypes.c_void_p, _D]
        L.orc_equilibrium_state.argtypes = [ctypes.c_void_p, _D]
        L.orc_eq_prim.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, _D]
        L.orc_coords.argtypes = [ctypes.c_void_p, ctypes.c_int, _D, _D]
        L.orc_metric.argtypes = [ctypes.c_void_p, ctypes.c_int, _D]
        L.orc_rhs.argtypes = [ctypes.c_void_p, _D, _D]
        L.orc_stage.argtypes = [ctypes.c_void_p, _D, _D, _D, ctypes.c_double, ctypes.c_double, ctypes.c_int]
        L.orc_step.argtypes = [ctypes.c_void_p, _D, ctypes.c_double, ctypes.c_double, ctypes.c_int]
        L.orc_step_tlm.argtypes = [ctypes.c_void_p, _D, _D, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_int]
        L.orc_step_sampled.argtypes = [ctypes.c_void_p, _D, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                       _L, ctypes.c_long, _D]
        L.orc_cfl_dt.restype = ctypes.c_double
        L.orc_cfl_dt.argtypes = [ctypes.c_void_p, _D]
        L.orc_sums.argtypes = [ctypes.c_void_p, _D, _D]
        L.orc_counters.argtypes = [ctypes.c_void_p, _L]
        L.orc_riemann.argtypes = [ctypes.c_double, _D, _D, ctypes.c_double, _D, _D]
        L.orc_parabola.argtypes = [ctypes.c_double] * 8 + [_D]
        L.orc_gas_flux.argtypes = [ctypes.c_void_p, ctypes.c_int, _D, _D, _D]
        L.orc_dust_flux.argtypes = [ctypes.c_int, _D, _D, _D]
        L.orc_drag.argtypes = [ctypes.c_void_p, ctypes.c_int, _D, ctypes.c_double, ctypes.c_double, ctypes.c_int]
        L.orc_status.argtypes = [ctypes.c_void_p]
        L.orc_set_indirect.argtypes = [ctypes.c_void_p, ctypes.c_double]
        L.orc_indirect.argtypes = [ctypes.c_void_p, _D, _D]
        L.orc_set_damping.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.orc_set_stokes_regime.argtypes = [ctypes.c_void_p, ctypes.c_double]
        L.orc_sources.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D]
        L.orc_set_species_stokes.argtypes = [ctypes.c_void_p, _D, ctypes.c_int]
        L.orc_set_recon.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_set_dust_recon.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_set_drag_scheme.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_set_vertical_damping.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double]
        L.orc_damping_rate.restype = ctypes.c_double
        L.orc_damping_rate.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
        L.orc_recon_faces.argtypes = [ctypes.c_void_p, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      _D, _D]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def riemann(gamma, WL, WR, S=0.0):
    """Exact Riemann solution sampled at x/t = S: ((rho, u, p), p*, u*, iters, converged, side, vacuum)."""
    wl = np.ascontiguousarray(WL, dtype=np.float64)
    wr = np.ascontiguousarray(WR, dtype=np.float64)
    W = np.zeros(3)
    star = np.zeros(5)
    vac = lib().orc_riemann(gamma, _p(wl), _p(wr), S, _p(W), _p(star))
    return W, star[0], star[1], int(star[2]), bool(star[3]), int(star[4]), bool(vac)


def parabola(em, e0, ep, xm, x0, xp, fm, fp):
    q = np.zeros(2)
    shaped = lib().orc_parabola(em, e0, ep, xm, x0, xp, fm, fp, _p(q))
    return q[0], q[1], bool(shaped)


def dust_flux(ax, UL, UR):
    ul = np.ascontiguousarray(UL, dtype=np.float64)
    ur = np.ascontiguousarray(UR, dtype=np.float64)
    F = np.zeros(4)
    lib().orc_dust_flux(ax, _p(ul), _p(ur), _p(F))
    return F


class Oracle:
    """One grid of the oracle; states are float64 arrays of shape (nf, nz, nth, nr)."""

    def __init__(self, w: syn.Workload):
        self.w = w
        d = _Desc(w.geometry, w.nr, w.nth, w.nz, (ctypes.c_double * 3)(*w.x0), (ctypes.c_double * 3)(*w.x1),
                  (ctypes.c_int * 3)(*w.bc_lo), (ctypes.c_int * 3)(*w.bc_hi),
                  w.gamma, w.gm, w.omega_frame, w.cfl, w.n_dust)
        self.h = ctypes.c_void_p(lib().orc_create(ctypes.byref(d)))
        self.nf = lib().orc_nfields(self.h)
        self.shape = (self.nf, w.nz, w.nth, w.nr)
        self.status = 0
        self.x_ind = 0.0
        self.drag_scheme = 0
        if lib().orc_set_recon(self.h, int(w.recon)):
            raise ValueError(f"unknown reconstruction mode {w.recon}")
        if w.drag_kappa:
            lib().orc_set_stokes_regime(self.h, float(w.drag_kappa))
        if w.dust_stokes_factors:
            self.set_species_stokes(w.dust_stokes_factors)
        if w.disc is not None:
            disc = np.array(w.disc_params(), dtype=np.float64)
            self.status |= lib().orc_set_equilibrium(self.h, _p(disc))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_destroy(self.h)
            self.h = None

    # ---- geometry / equilibrium
    def coords(self, ax):
        n = (self.w.nr, self.w.nth, self.w.nz)[ax]
        c = np.zeros(n + 6)
        f = np.zeros(n + 7)
        lib().orc_coords(self.h, ax, _p(c), _p(f))
        return c[3:-3], f[3:-3]

    def metric(self, i):
        m = np.zeros(8)
        lib().orc_metric(self.h, i, _p(m))
        return m

    def volumes(self):
        return np.array([self.metric(i)[0] for i in range(self.w.nr)])

    def eq_prim(self, r, z):
        out = np.zeros(3)
        lib().orc_eq_prim(self.h, r, z, _p(out))
        return out

    def equilibrium_state(self):
        E = np.zeros(self.shape)
        lib().orc_equilibrium_state(self.h, _p(E))
        return E

    # ---- the method
    def set_indirect(self, x_ref):
        """X_ref of the indirect-gravity term (Sect. 2.10); 0 switches it off."""
        self.x_ind = float(x_ref)
        lib().orc_set_indirect(self.h, self.x_ind)

    def set_dust_recon(self, mode):
        """Dust reconstruction (reading R5): 0 = the parabola on rho_d and the
        velocity (the default), 1 = the velocity flat in a cell where rho_d is
        a local maximum and the flow converges along the axis."""
        if lib().orc_set_dust_recon(self.h, int(mode)):
            raise ValueError(f"unknown dust reconstruction mode {mode}")

    def set_drag_scheme(self, mode):
        """Drag integration (reading R7): 0 = backward Euler in closed form
        after each RK2 stage (the default), 1 = Strang splitting, half a step
        of trapezoidal drag before and after the RK2 step of the other terms.
        Single stages and sampled steps follow the default only."""
        if lib().orc_set_drag_scheme(self.h, int(mode)):
            raise ValueError(f"unknown drag scheme {mode}")
        self.drag_scheme = int(mode)

    def set_damping(self, r_ein, r_eout, period_factor=1.0):
        """Wave-killing zones r < r_ein and r > r_eout (reading R17); a
        period_factor <= 0 switches them off."""
        if lib().orc_set_damping(self.h, float(r_ein), float(r_eout), float(period_factor)):
            raise ValueError("damping zones must lie inside the radial extent of a cylindrical grid")

    def set_vertical_damping(self, z_edge, period_factor=1.0):
        """Vertical sheared damped boundary (reading R21): relaxation in
        |z| > z_edge; a period_factor <= 0 switches it off."""
        if lib().orc_set_vertical_damping(self.h, float(z_edge), float(period_factor)):
            raise ValueError("the vertical zone must lie inside a cylindrical grid symmetric about z = 0")

    def damping_rate(self, i, k):
        """Relaxation rate of the damping zones at cell (i, k) (R17 + R21)."""
        return lib().orc_damping_rate(self.h, int(i), int(k))

    def sources(self, i, j, k, U):
        """App. B source vector per unit volume of the state U at cell (i, j, k)."""
        U = np.ascontiguousarray(U, dtype=np.float64)
        S = np.zeros(self.nf)
        lib().orc_sources(self.h, i, j, k, _p(U), _p(S))
        return S

    def set_species_stokes(self, factors):
        """Stokes-number factors of the dust species (species 0 keeps St)."""
        f = np.ascontiguousarray(factors, dtype=np.float64)
        lib().orc_set_species_stokes(self.h, _p(f), len(f))

    def set_stokes_regime(self, kappa):
        """kappa = r_p / lambda_0 of drag law 2 (reading R19); <= 0: Epstein only."""
        lib().orc_set_stokes_regime(self.h, float(kappa))

    def indirect(self, E):
        """X_ref (A_disc, B_disc) of the state E (Sect. 2.10)."""
        E = np.ascontiguousarray(E, dtype=np.float64)
        out = np.zeros(2)
        lib().orc_indirect(self.h, _p(E), _p(out))
        return out

    def recon_faces(self, E, ax, i, j, k):
        """Full reconstructed states (E0 + q) on the lower and upper faces of
        cell (i, j, k) along axis ax (Sect. 2.7): (Um, Up), nf values each."""
        E = np.ascontiguousarray(E, dtype=np.float64)
        Um = np.zeros(self.nf)
        Up = np.zeros(self.nf)
        lib().orc_recon_faces(self.h, _p(E), ax, i, j, k, _p(Um), _p(Up))
        return Um, Up

    def rhs(self, E):
        E = np.ascontiguousarray(E, dtype=np.float64)
        G = np.zeros_like(E)
        self.status |= lib().orc_rhs(self.h, _p(E), _p(G))
        return G

    def stage(self, Ein, Ebase, tau):
        if self.drag_scheme:
            raise ValueError("single stages follow the default drag integration")
        Ein = np.ascontiguousarray(Ein, dtype=np.float64)
        Ebase = np.ascontiguousarray(Ebase, dtype=np.float64)
        out = np.zeros_like(Ein)
        self.status |= lib().orc_stage(self.h, _p(Ein), _p(Ebase), _p(out), tau, self.w.stokes, self.w.drag_law)
        return out

    def step(self, E, dt):
        """One RK2 step; returns a new array."""
        E = np.array(E, dtype=np.float64, order="C", copy=True)
        self.status |= lib().orc_step(self.h, _p(E), dt, self.w.stokes, self.w.drag_law)
        return E

    def step_tlm(self, E, dE, dt, dstokes=0.0, stokes=None):
        """Tangent-linear RK2 step at fixed dt: returns (E^{n+1}, dE^{n+1}) for the
        direction (dE, dstokes); Stokes number defaults to the workload's."""
        E = np.array(E, dtype=np.float64, order="C", copy=True)
        dE = np.array(dE, dtype=np.float64, order="C", copy=True)
        st = self.w.stokes if stokes is None else stokes
        self.status |= lib().orc_step_tlm(self.h, _p(E), _p(dE), dt, st, dstokes, self.w.drag_law)
        return E, dE

    def step_sampled(self, E, dt, cells):
        if self.x_ind != 0.0:
            raise ValueError("sampled steps need the whole stage state when indirect gravity is on")
        if self.drag_scheme:
            raise ValueError("sampled steps follow the default drag integration")
        E = np.ascontiguousarray(E, dtype=np.float64)
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        out = np.zeros((len(cells), self.nf))
        self.status |= lib().orc_step_sampled(self.h, _p(E), dt, self.w.stokes, self.w.drag_law,
                                              cells.ctypes.data_as(_L), len(cells), _p(out))
        return out

    def cfl_dt(self, E):
        E = np.ascontiguousarray(E, dtype=np.float64)
        return lib().orc_cfl_dt(self.h, _p(E))

    def sums(self, E):
        E = np.ascontiguousarray(E, dtype=np.float64)
        s = np.zeros(self.nf)
        lib().orc_sums(self.h, _p(E), _p(s))
        return s

    def gas_flux(self, ax, UL, UR):
        ul = np.ascontiguousarray(UL, dtype=np.float64)
        ur = np.ascontiguousarray(UR, dtype=np.float64)
        F = np.zeros(5)
        lib().orc_gas_flux(self.h, ax, _p(ul), _p(ur), _p(F))
        return F

    def drag(self, i, U, tau):
        U = np.array(U, dtype=np.float64, copy=True)
        lib().orc_drag(self.h, i, _p(U), tau, self.w.stokes, self.w.drag_law)
        return U

    def counters(self):
        c = np.zeros(2, dtype=np.int64)
        lib().orc_counters(self.h, c.ctypes.data_as(_L))
        return c

    def take_status(self):
        s = self.status | lib().orc_status(self.h)
        self.status = 0
        return s

    # ---- runs
    def run(self, E, steps=None, t_end=None, dts=None):
        """Advance with the CFL step (or the given dt list); returns (E, t, dts)."""
        t = 0.0
        used = []
        if dts is not None:
            for dt in dts:
                E = self.step(E, dt)
                t += dt
                used.append(dt)
            return E, t, used
        n = 0
        while True:
            if steps is not None and n >= steps:
                break
            dt = self.cfl_dt(E)
            if t_end is not None:
                if t >= t_end * (1 - 1e-14):
                    break
                dt = min(dt, t_end - t)
            E = self.step(E, dt)
            t += dt
            used.append(dt)
            n += 1
        return E, t, used


# ---------------------------------------------------------------- initial conditions (oracle side)
def initial_state(o: Oracle) -> np.ndarray:
    """Full conservative initial state (nf, nz, nth, nr) for the workload, built on the oracle's
    own equilibrium; the recipe is the one stated for each workload."""
    w = o.w
    nf = o.nf
    g = w.gamma
    E = np.zeros(o.shape)
    if w.ic == "sod":
        xc, _ = o.coords(0)
        left = xc < 0.5
        rho = np.where(left, 1.0, 0.125)
        p = np.where(left, 1.0, 0.1)
        E[syn.F_RHO] = rho[None, None, :]
        E[syn.F_EN] = (p / (g - 1.0))[None, None, :]
        return E
    if w.ic == "explosion":  # Sect. 4.1: (rho, P) = (1, 1) for r <= 0.4, (0.125, 0.1) outside, at rest
        rc, _ = o.coords(0)
        inside = rc <= 0.4
        E[syn.F_RHO] = np.where(inside, 1.0, 0.125)[None, None, :]
        E[syn.F_EN] = (np.where(inside, 1.0, 0.1) / (g - 1.0))[None, None, :]
        return E
    E0 = o.equilibrium_state()
    rho0 = E0[syn.F_RHO]
    v0 = E0[syn.F_MV] / rho0
    E[:5] = E0[:5]
    if w.ic == "noise":
        xi = syn.uniform_pm1(w.seed, syn.F_RHO, w.ncell).reshape(w.nz, w.nth, w.nr)
        drho = w.noise_amp * xi * rho0
        E[syn.F_RHO] += drho
        E[syn.F_MV] += drho * v0
        E[syn.F_EN] += 0.5 * drho * v0 * v0
    elif w.ic == "vortex":
        r, _ = o.coords(0)
        th, _ = o.coords(1)
        R = r[None, None, :]
        TH = th[None, :, None]
        up = np.zeros((1, w.nth, w.nr))
        vp = np.zeros((1, w.nth, w.nr))
        for (rv, thv) in w.vortices:
            sig_r = w.vortex_width_h * math.sqrt(2.0 * w.disc[2] * rv ** w.disc[3]) / math.sqrt(w.gm / rv ** 3)
            sig_t = w.vortex_chi * sig_r
            omega_c = -w.vortex_amp * 1.5 * math.sqrt(w.gm / rv ** 3)
            psi0 = omega_c / (1.0 / sig_r ** 2 + 1.0 / sig_t ** 2)
            dth = np.mod(TH - thv + math.pi, 2.0 * math.pi) - math.pi
            psi = psi0 * np.exp(-(R - rv) ** 2 / (2.0 * sig_r ** 2) - (rv * dth) ** 2 / (2.0 * sig_t ** 2))
            up += -psi * rv * rv * dth / (R * sig_t ** 2)        # (1/r) dpsi/dtheta
            vp += psi * (R - rv) / sig_r ** 2                     # -dpsi/dr
        E[syn.F_MU] = rho0 * up
        E[syn.F_MV] += rho0 * vp
        E[syn.F_EN] += 0.5 * rho0 * (up * up + 2.0 * v0 * vp + vp * vp)
        nd = (nf - 5) // 4
        for s in range(nd):  # each species: its share of the dust, its own noise, moving with the gas
            b = 5 + 4 * s
            xi = syn.uniform_pm1(w.seed, syn.F_DRHO + 4 * s, w.ncell).reshape(w.nz, w.nth, w.nr)
            rd = w.dust_ratio / nd * rho0 * (1.0 + w.dust_noise * xi)
            E[b + 3] = rd
            E[b] = rd * up
            E[b + 1] = rd * (v0 + vp)
            E[b + 2] = 0.0
    elif w.ic == "rwi":  # Sect. 4.3: the bumped equilibrium (reading R22), seeded v_r of mode m
        r, _ = o.coords(0)
        th, _ = o.coords(1)
        z, _ = o.coords(2)
        G = np.exp(-((r - w.rwi_r0) / (math.sqrt(2.0) * w.rwi_width)) ** 2)[None, None, :]
        vth0 = np.array([[o.eq_prim(ri, zk)[1] for ri in r] for zk in z])[:, None, :]  # inertial v_theta0
        vr = w.rwi_eps * vth0 * np.sin(w.rwi_mode * th)[None, :, None] * G
        E[syn.F_MU] = rho0 * vr
        E[syn.F_EN] += 0.5 * rho0 * vr * vr
    else:
        raise ValueError(w.ic)
    return E
