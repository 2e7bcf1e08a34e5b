"""Pins of the oracle on the cylindrical explosion test (Sect. 4.1).

The explosion is a 2-D Riemann problem with cylindrical symmetry: its exact
solution depends on r and t only and obeys the 1-D Euler equations with the
geometric source of the polar mesh, d(rU)/dt + d(rF)/dr = (0, P, 0).  Toro
(ch. 17) takes a converged 1-D solution of those equations as the reference.
The test writes its own 1-D solver for them, independent of the oracle in
every part (uniform mesh from the axis with a reflecting axis, primitive
MUSCL reconstruction with minmod, HLL flux, Heun time stepping), runs it on a
fine mesh, and checks that the oracle's 2-D solution on the logarithmic polar
mesh converges to it.  Further pins: the solution stays exactly independent
of theta, and a uniform gas at rest shows the closed-form residual of the
centre-point pressure source on the logarithmic mesh (reading R1), which
the balanced scheme removes from disc runs but which the explosion, having
no equilibrium, keeps (velocities ~2e-4 ahead of the waves at 80 cells).
"""
import os

import numpy as np
import pytest

import oracle
import synthetic as syn

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "explosion_sect4_1.txt")

GAMMA = 1.4
T_END = 0.25


def _radial_reference(n=2000, r_max=1.0, t_end=T_END, cfl=0.4):
    """1-D cylindrically symmetric Euler solution on [0, r_max]: finite
    volumes of the annuli, HLL fluxes of MUSCL (minmod) primitive states,
    two-stage Heun steps; reflecting axis at r = 0, zero-gradient outer edge.
    Returns cell centres and (rho, u, P)."""
    dr = r_max / n
    rf = np.arange(n + 1) * dr
    rc = 0.5 * (rf[:-1] + rf[1:])
    area = rf                       # face "area" per radian and unit height
    vol = 0.5 * (rf[1:] ** 2 - rf[:-1] ** 2)
    rho = np.where(rc <= 0.4, 1.0, 0.125)
    p = np.where(rc <= 0.4, 1.0, 0.1)
    U = np.stack([rho, np.zeros(n), p / (GAMMA - 1.0)])

    def prim(U):
        rho = U[0]
        u = U[1] / rho
        return rho, u, (GAMMA - 1.0) * (U[2] - 0.5 * rho * u * u)

    def minmod(a, b):
        return np.where(a * b > 0.0, np.sign(a) * np.minimum(np.abs(a), np.abs(b)), 0.0)

    def rhs(U):
        rho, u, p = prim(U)
        W = np.stack([rho, u, p])
        # two ghost cells each side: mirror (u -> -u) at the axis, copy outside
        Wg = np.concatenate([W[:, 1::-1] * np.array([[1], [-1], [1]]), W, W[:, -1:], W[:, -1:]], axis=1)
        s = minmod(Wg[:, 1:-1] - Wg[:, :-2], Wg[:, 2:] - Wg[:, 1:-1])   # slopes of cells -1..n
        WL = Wg[:, 1:-2] + 0.5 * s[:, :-1]                              # faces 0..n, left state
        WR = Wg[:, 2:-1] - 0.5 * s[:, 1:]                               # right state

        def flux(W):
            rho, u, p = W
            E = p / (GAMMA - 1.0) + 0.5 * rho * u * u
            return np.stack([rho * u, rho * u * u + p, u * (E + p)]), np.stack([rho, rho * u, E])

        FL, UL = flux(WL)
        FR, UR = flux(WR)
        cL = np.sqrt(GAMMA * WL[2] / WL[0])
        cR = np.sqrt(GAMMA * WR[2] / WR[0])
        sL = np.minimum(WL[1] - cL, WR[1] - cR)
        sR = np.maximum(WL[1] + cL, WR[1] + cR)
        F = np.where(sL >= 0, FL, np.where(sR <= 0, FR, (sR * FL - sL * FR + sL * sR * (UR - UL)) / (sR - sL)))
        F[:, 0] = 0.0
        F[1, 0] = WL[2, 0]  # the axis face has zero area; momentum flux there is P, times area 0
        G = -(area[1:] * F[:, 1:] - area[:-1] * F[:, :-1])
        G[1] += p * dr      # geometric source: integral of P/r over the annulus, times r
        return G / vol, np.max(np.abs(u) + np.sqrt(GAMMA * p / rho))

    t = 0.0
    while t < t_end:
        k1, amax = rhs(U)
        dt = min(cfl * dr / amax, t_end - t)
        U1 = U + dt * k1
        k2, _ = rhs(U1)
        U = 0.5 * (U + U1 + dt * k2)
        t += dt
    return rc, prim(U)


@pytest.fixture(scope="module")
def reference():
    return _radial_reference()


def _oracle_run(nr, nth=4, t_end=T_END):
    w = syn.scaled(syn.EXPLOSION, nr, nth, 1, t_end=t_end)
    o = oracle.Oracle(w)
    E0 = oracle.initial_state(o)
    E, t, dts = o.run(E0.copy(), t_end=t_end)
    assert o.take_status() == 0 and t == pytest.approx(t_end, rel=1e-14)
    return w, o, E0, E, dts


def test_reference_solver_conserves_mass():
    """The 1-D reference itself: mass is conserved (no wave reaches r = 1)."""
    rc, (rho, u, p) = _radial_reference(n=400)
    r0 = np.where(rc <= 0.4, 1.0, 0.125)
    assert abs((rho * rc).sum() - (r0 * rc).sum()) <= 1e-12 * (r0 * rc).sum()


def test_explosion_converges_to_the_radial_solution(reference):
    rr, (rho_ref, u_ref, p_ref) = reference
    errs = {}
    for nr in (100, 200):
        w, o, E0, E, _ = _oracle_run(nr)
        rc, _ = o.coords(0)
        V = o.volumes()
        rho = E[4, 0, 0]
        u = E[0, 0, 0] / rho
        ref = np.interp(rc, rr, rho_ref)
        errs[nr] = (V * np.abs(rho - ref)).sum() / (V * ref).sum()
        # the velocity field is radial: no azimuthal or vertical momentum appears
        assert not E[1].any() and not E[2].any()
        assert np.abs(u - np.interp(rc, rr, u_ref)).max() < 0.5
    print("explosion density L1 vs the radial reference:", errs)
    assert errs[200] < 0.03, errs
    assert errs[200] < 0.7 * errs[100], errs


def test_explosion_keeps_cylindrical_symmetry_exactly():
    w, o, E0, E, _ = _oracle_run(60, nth=8, t_end=0.1)
    assert np.array_equal(E, np.broadcast_to(E[:, :, :1, :], E.shape))


def test_uniform_gas_at_rest_feels_the_closed_form_imbalance():
    """A uniform gas at rest on the polar mesh: the radial momentum residual
    of a cell is the pressure source at the centre minus the face-area
    difference, G = P dtheta dz ((r+^2 - r-^2) / (2 r_c) - (r+ - r-)), with
    r_c = sqrt(r+ r-) (reading R1); with the balanced scheme of Sect. 2.8 a
    disc never sees it, the explosion (no equilibrium) does.  Every other
    field's residual is zero."""
    w = syn.scaled(syn.EXPLOSION, 40, 8, 1)
    o = oracle.Oracle(w)
    E = np.zeros(o.shape)
    E[4] = 1.0
    E[3] = 2.0 / (GAMMA - 1.0)   # P = 2
    G = o.rhs(E)
    assert o.take_status() == 0
    _, rf = o.coords(0)
    rm, rp = rf[:-1], rf[1:]
    dth = 2.0 * np.pi / w.nth
    dz = w.x1[2] - w.x0[2]
    ref = 2.0 * dth * dz * ((rp * rp - rm * rm) / (2.0 * np.sqrt(rp * rm)) - (rp - rm))
    assert np.allclose(G[0], ref[None, None, :], rtol=1e-9, atol=0)
    assert (ref > 0).all()  # the geometric-mean centre makes the source win
    for f in (1, 2, 3, 4):
        assert np.abs(G[f]).max() <= 1e-14 * np.abs(ref).max(), f


def test_workload_is_the_papers_explosion():
    """The workload and the oracle's initial state carry the values printed in
    Sect. 4.1 (tests/golden/explosion_sect4_1.txt)."""
    gold = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            k, *v = line.split()
            gold[k] = v
    w = syn.EXPLOSION
    assert w.gamma == float(gold["gamma"][0])
    assert (w.nr, w.nth) == (int(gold["N_r"][0]), int(gold["N_theta"][0]))
    ws = syn.scaled(w, 64, 4, 1)
    o = oracle.Oracle(ws)
    E = oracle.initial_state(o)
    rc, _ = o.coords(0)
    r_d = float(gold["r_diaphragm"][0])
    for side, sel in (("inside", rc <= r_d), ("outside", rc > r_d)):
        vals = dict(zip(gold[side][::2], map(float, gold[side][1::2])))
        rho = E[4][..., sel]
        assert np.all(rho == vals["rho"])
        assert np.all(E[0][..., sel] == vals["v_r"] * rho) and np.all(E[1][..., sel] == vals["v_theta"] * rho)
        assert np.allclose((w.gamma - 1.0) * E[3][..., sel], vals["P"], rtol=1e-15, atol=0)
