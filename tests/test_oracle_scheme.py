"""Pins of the oracle's whole time step.

- Balanced scheme (Sect. 2.8): the disc equilibrium is reproduced bit-exactly
  step after step (the paper reports < 1e-9 after 300 orbits).
- Conservation (Sect. 2.2 finite-volume form): in a periodic Box the volume sums
  of mass, momentum and energy are constant to round-off; with dust and drag
  the total (gas + dust) momentum is.
- Sod shock tube (the Box workload) converges to the exact Riemann solution,
  whose solver is pinned separately.
- Axis permutation and mirror symmetry of the Sod problem catch index, sign and
  transposition mistakes in the directional sweeps.
- Drag (Sect. 2.9, semi-implicit reading): closed-form relaxation in a uniform
  Box; CFL (Sect. 2.5): closed form on a uniform state.
- Dust flux (Sect. 2.9, kinetic flux-splitting reading): its case table.
- Rotating-frame sources: the radial-momentum response to an azimuthal velocity
  perturbation is 2 rho v_theta dv / r + rho dv^2 / r in both frames.
"""
import numpy as np
import pytest

import oracle
import synthetic as syn


def _box(n=(16, 8, 8), n_dust=0, stokes=0.0):
    L = (1.0, n[1] / n[0], n[2] / n[0])
    return syn.Workload(name="box", geometry=syn.GEOM_BOX, nr=n[0], nth=n[1], nz=n[2], x0=(0.0, 0.0, 0.0), x1=L,
                        bc_lo=(0, 0, 0), bc_hi=(0, 0, 0), ic="none", steps=0, omega_frame=0.0, n_dust=n_dust,
                        stokes=stokes)


def _smooth_box_state(o, seed=3):
    w = o.w
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(*(np.arange(n) / n for n in (w.nz, w.nth, w.nr)), indexing="ij")
    E = np.zeros(o.shape)
    rho = 1.0 + 0.2 * np.sin(2 * np.pi * (x + rng.uniform())) * np.cos(2 * np.pi * (y + rng.uniform()))
    u = 0.3 * np.cos(2 * np.pi * (x + z))
    v = -0.2 + 0.1 * np.sin(2 * np.pi * y)
    ww = 0.1 * np.sin(2 * np.pi * (z + x))
    p = 1.0 + 0.3 * np.cos(2 * np.pi * (y + z))
    E[syn.F_RHO] = rho
    E[syn.F_MU], E[syn.F_MV], E[syn.F_MW] = rho * u, rho * v, rho * ww
    E[syn.F_EN] = 0.5 * rho * (u * u + v * v + ww * ww) + p / (w.gamma - 1)
    if o.nf > 5:
        rd = 0.5 + 0.3 * np.cos(2 * np.pi * (x - y))
        E[syn.F_DRHO] = rd
        E[syn.F_DMU], E[syn.F_DMV], E[syn.F_DMW] = rd * (u + 0.2), rd * v, rd * (ww - 0.1)
    return E


@pytest.mark.parametrize("n_dust", [0, 1])
def test_equilibrium_bit_exact(n_dust):
    w = syn.scaled(syn.DISC_NOISE, 12, 8, 32, steps=4, n_dust=n_dust, stokes=0.1)
    o = oracle.Oracle(w)
    E0 = o.equilibrium_state()
    E, _, dts = o.run(E0.copy(), steps=4)
    assert o.take_status() == 0
    assert np.array_equal(E, E0)


@pytest.mark.parametrize("n_dust,stokes", [(0, 0.0), (1, 0.05)])
def test_box_conservation(n_dust, stokes):
    o = oracle.Oracle(_box(n_dust=n_dust, stokes=stokes))
    E = _smooth_box_state(o)
    s0 = o.sums(E)
    E, _, _ = o.run(E, steps=12)
    assert o.take_status() == 0
    s1 = o.sums(E)
    V = o.volumes()[0]
    scale = np.abs(E).sum(axis=(1, 2, 3)) * V
    if n_dust == 0:
        assert np.all(np.abs(s1 - s0) <= 1e-14 * scale * 12)
    else:
        for f in (syn.F_RHO, syn.F_DRHO):  # both masses
            assert abs(s1[f] - s0[f]) <= 1e-14 * scale[f] * 12
        for c in range(3):  # total momentum
            tot0 = s0[syn.F_MU + c] + s0[syn.F_DMU + c]
            tot1 = s1[syn.F_MU + c] + s1[syn.F_DMU + c]
            assert abs(tot1 - tot0) <= 1e-14 * (scale[syn.F_MU + c] + scale[syn.F_DMU + c]) * 12


def _sod_profile(nr, axis=0, mirror=False, recon=syn.RECON_CONSERVATIVE):
    n = [4, 4, 4]
    n[axis] = nr
    L = [4.0 / nr] * 3
    L[axis] = 1.0
    bc_lo = [syn.BC_PERIODIC] * 3
    bc_hi = [syn.BC_PERIODIC] * 3
    bc_lo[axis] = bc_hi[axis] = syn.BC_OUTFLOW
    w = syn.Workload(name="sod", geometry=syn.GEOM_BOX, nr=n[0], nth=n[1], nz=n[2], x0=(0, 0, 0), x1=tuple(L),
                     bc_lo=tuple(bc_lo), bc_hi=tuple(bc_hi), ic="none", steps=0, omega_frame=0.0, recon=recon)
    o = oracle.Oracle(w)
    xc, _ = o.coords(axis)
    left = xc < 0.5
    if mirror:
        left = ~left
    shape = [1, 1, 1]
    shape[2 - axis] = nr
    E = np.zeros(o.shape)
    rho = np.where(left, 1.0, 0.125).reshape(shape)
    p = np.where(left, 1.0, 0.1).reshape(shape)
    E[syn.F_RHO] = np.broadcast_to(rho, o.shape[1:])
    E[syn.F_EN] = np.broadcast_to(p / 0.4, o.shape[1:])
    E, t, _ = o.run(E, t_end=0.2)
    assert o.take_status() == 0 and t == pytest.approx(0.2, rel=1e-14)
    mom = (syn.F_MU, syn.F_MV, syn.F_MW)[axis]
    line = [0, 0, 0]
    sl = [slice(0, 1)] * 3
    sl[2 - axis] = slice(None)
    rho_line = E[syn.F_RHO][tuple(sl)].ravel()
    m_line = E[mom][tuple(sl)].ravel()
    return xc, rho_line, m_line


@pytest.mark.parametrize("recon", [syn.RECON_CONSERVATIVE, syn.RECON_PRIMITIVE, syn.RECON_PRESSURE],
                         ids=["conservative", "primitive", "pressure"])
def test_sod_converges_to_exact(recon):
    errs = []
    for nr in (128, 256):
        xc, rho, _ = _sod_profile(nr, recon=recon)
        exact = np.array([oracle.riemann(1.4, (1, 0, 1), (0.125, 0, 0.1), S=(x - 0.5) / 0.2)[0][0] for x in xc])
        errs.append(np.abs(rho - exact).mean())
    print("Sod L1 density errors at 128 and 256 cells", [f"{e:.2e}" for e in errs])
    assert errs[1] < 0.75 * errs[0]
    assert errs[1] < 0.01


@pytest.mark.parametrize("axis", [1, 2])
def test_sod_axis_permutation(axis):
    _, rho_x, m_x = _sod_profile(64, axis=0)
    _, rho_a, m_a = _sod_profile(64, axis=axis)
    np.testing.assert_allclose(rho_a, rho_x, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(m_a, m_x, rtol=1e-13, atol=1e-14)


def test_sod_mirror_symmetry():
    _, rho, m = _sod_profile(64)
    _, rho_m, m_m = _sod_profile(64, mirror=True)
    np.testing.assert_allclose(rho_m[::-1], rho, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(-m_m[::-1], m, rtol=1e-13, atol=1e-13)


def test_drag_closed_form():
    """Uniform gas and dust with a velocity offset: G vanishes, so each step is the
    backward-Euler relaxation over dt of the relative velocity."""
    St = 0.3
    o = oracle.Oracle(_box(n=(4, 4, 4), n_dust=1, stokes=St))
    E = np.zeros(o.shape)
    rg, rd = 1.0, 0.4
    vg, vd = np.array([0.1, -0.2, 0.05]), np.array([0.5, 0.3, -0.25])
    p = 1.0
    E[syn.F_RHO], E[syn.F_DRHO] = rg, rd
    for c in range(3):
        E[syn.F_MU + c] = rg * vg[c]
        E[syn.F_DMU + c] = rd * vd[c]
    E[syn.F_EN] = 0.5 * rg * vg @ vg + p / 0.4
    dts = [0.01, 0.02, 0.05, 0.1]
    E1, _, _ = o.run(E, dts=dts)
    eps = rd / rg
    factor = np.prod([1.0 / (1.0 + dt * (1 + eps) / St) for dt in dts])
    dv0 = vd - vg
    vg1 = E1[syn.F_MU:syn.F_MU + 3, 0, 0, 0] / rg
    vd1 = E1[syn.F_DMU:syn.F_DMU + 3, 0, 0, 0] / rd
    np.testing.assert_allclose(vd1 - vg1, dv0 * factor, rtol=1e-13)
    np.testing.assert_allclose(rg * vg1 + rd * vd1, rg * vg + rd * vd, rtol=1e-14, atol=1e-15)
    # gas internal energy unchanged: the drag only does work on the gas bulk motion
    P1 = 0.4 * (E1[syn.F_EN, 0, 0, 0] - 0.5 * rg * vg1 @ vg1)
    assert P1 == pytest.approx(p, rel=1e-13)
    # first-order approach to the continuous relaxation exp(-(1+eps) t / St)
    o2 = oracle.Oracle(_box(n=(4, 4, 4), n_dust=1, stokes=St))
    errs = []
    for nsub in (50, 100):
        E2, _, _ = o2.run(E, dts=[0.2 / nsub] * nsub)
        dv = E2[syn.F_DMU, 0, 0, 0] / rd - E2[syn.F_MU, 0, 0, 0] / rg
        errs.append(abs(dv - dv0[0] * np.exp(-(1 + eps) * 0.2 / St)))
    assert errs[1] < 0.55 * errs[0]


def test_cfl_closed_form():
    o = oracle.Oracle(_box(n=(16, 16, 16)))
    E = np.zeros(o.shape)
    rho, u, v, w, p = 1.3, 0.4, -0.3, 0.2, 0.9
    E[syn.F_RHO] = rho
    E[syn.F_MU], E[syn.F_MV], E[syn.F_MW] = rho * u, rho * v, rho * w
    E[syn.F_EN] = 0.5 * rho * (u * u + v * v + w * w) + p / 0.4
    dx = 1.0 / 16
    expect = 0.5 * dx / (np.sqrt(u * u + v * v + w * w) + np.sqrt(1.4 * p / rho))
    assert o.cfl_dt(E) == pytest.approx(expect, rel=1e-14)


@pytest.mark.parametrize("ul,ur,pick", [(0.5, 0.3, "L"), (-0.5, -0.3, "R"), (-0.2, 0.4, "0"), (0.0, 0.0, "0"),
                                        (0.6, -0.2, "LR"), (0.2, -0.6, "LR"), (0.3, 0.0, "L"), (0.0, -0.4, "R")])
def test_dust_flux_cases(ul, ur, pick):
    """Matter moving right crosses the face from the left state, matter moving
    left from the right state; converging streams both cross (a delta shock
    accumulates mass), diverging streams leave the face empty."""
    rl, rr = 2.0, 0.5
    UL = np.array([rl * ul, rl * 0.1, rl * -0.2, rl])  # x-direction: (rho u, rho v, rho w, rho)
    UR = np.array([rr * ur, rr * 0.3, rr * 0.4, rr])
    F = oracle.dust_flux(0, UL, UR)
    FL = np.array([rl * ul * ul, rl * ul * 0.1, rl * ul * -0.2, rl * ul])
    FR = np.array([rr * ur * ur, rr * ur * 0.3, rr * ur * 0.4, rr * ur])
    expect = {"L": FL, "R": FR, "0": np.zeros(4), "LR": FL + FR}[pick]
    np.testing.assert_allclose(F, expect, rtol=1e-15, atol=1e-16)


def test_sampled_step_matches_full_step():
    w = syn.scaled(syn.VORTEX, 10, 12, 32, steps=1)
    o = oracle.Oracle(w)
    E = oracle.initial_state(o)
    dt = o.cfl_dt(E)
    full = o.step(E, dt)
    rng = np.random.default_rng(1)
    cells = np.concatenate([[0, w.ncell - 1, w.nr - 1], rng.integers(0, w.ncell, 20)])
    samp = o.step_sampled(E, dt, cells)
    np.testing.assert_array_equal(samp, full.reshape(o.nf, -1)[:, cells].T)


@pytest.mark.parametrize("omega", [0.0, 1.0])
def test_rotating_frame_radial_response(omega):
    w = syn.scaled(syn.DISC_NOISE, 24, 4, 32, steps=1, omega_frame=omega)
    o = oracle.Oracle(w)
    E0 = o.equilibrium_state()
    dv = 1e-3
    E = E0.copy()
    rho = E0[syn.F_RHO]
    v0 = E0[syn.F_MV] / rho
    E[syn.F_MV] += rho * dv
    E[syn.F_EN] += rho * v0 * dv + 0.5 * rho * dv * dv
    G = o.rhs(E)
    rc, _ = o.coords(0)
    V = o.volumes()
    k, i = 16, 12
    _, vth, _ = o.eq_prim(rc[i], o.coords(2)[0][k])
    expect = (2.0 * rho[k, 0, i] * vth * dv + rho[k, 0, i] * dv * dv) / rc[i]
    assert G[syn.F_MU, k, 0, i] / V[i] == pytest.approx(expect, rel=2e-3)
