"""Pins of the oracle's parabolic reconstruction (Sect. 2.7) and of the disc
equilibrium (App. A).

Reconstruction: the three-point parabola is exact on quadratic profiles on a
non-uniform (logarithmic) mesh wherever the limiter leaves it alone, flat at an
extremum, bounded by the minmod slope times twice the face distance (at most
the neighbour distance) on an overshoot, never creates a
new extremum, and depends continuously (Lipschitz) on the cell values.
Equilibrium: central finite differences of the analytic P0 reproduce vertical
hydrostatic balance and radial centrifugal balance, and the column integral of
rho0 is the surface density Sigma(r) up to the O(h^2) spherical-potential
correction.
"""
import math

import numpy as np
import pytest

import oracle
import synthetic as syn


def _log_mesh(n=12, r0=0.5, r1=2.0):
    faces = r0 * (r1 / r0) ** (np.arange(n + 1) / n)
    centres = np.sqrt(faces[:-1] * faces[1:])
    return centres, faces


@pytest.mark.parametrize("coef", [(0.3, 1.0, 2.0), (-0.2, -1.5, 0.7), (0.0, 2.0, -1.0)])
def test_quadratic_exact(coef):
    a, b, c = coef
    xc, xf = _log_mesh()
    f = lambda x: a * x * x + b * x + c
    checked = 0
    for i in range(1, len(xc) - 1):
        qm, qp, shaped = oracle.parabola(f(xc[i - 1]), f(xc[i]), f(xc[i + 1]), xc[i - 1], xc[i], xc[i + 1],
                                         xf[i], xf[i + 1])
        vals = [f(xc[i - 1]), f(xc[i]), f(xc[i + 1])]
        sm = (vals[1] - vals[0]) / (xc[i] - xc[i - 1])
        sp = (vals[2] - vals[1]) / (xc[i + 1] - xc[i])
        smin = min(abs(sm), abs(sp)) if sm * sp > 0 else 0.0
        dm, dp = f(xf[i]) - vals[1], f(xf[i + 1]) - vals[1]
        # where each face deviation has the slope's sign and stays within twice the
        # minmod slope times the face distance, the limiter leaves the parabola alone
        hm = min(2 * (xc[i] - xf[i]), xc[i] - xc[i - 1])
        hp = min(2 * (xf[i + 1] - xc[i]), xc[i + 1] - xc[i])
        inside = smin > 0 and dm * sm < 0 and dp * sp > 0 and \
            abs(dm) < smin * hm * (1 - 1e-12) and abs(dp) < smin * hp * (1 - 1e-12)
        if inside:
            assert shaped
            assert qm == pytest.approx(f(xf[i]), rel=1e-13, abs=1e-13)
            assert qp == pytest.approx(f(xf[i + 1]), rel=1e-13, abs=1e-13)
            checked += 1
    assert checked >= 5


def test_extremum_is_flat():
    qm, qp, shaped = oracle.parabola(1.0, 2.0, 1.5, 0.0, 1.0, 2.0, 0.5, 1.5)
    assert not shaped and qm == 2.0 and qp == 2.0
    qm, qp, shaped = oracle.parabola(1.0, 1.0, 3.0, 0.0, 1.0, 2.0, 0.5, 1.5)  # zero slope on one side
    assert not shaped and qm == 1.0 and qp == 1.0


def test_overshoot_limited_by_minmod_bound():
    # slopes 1 and 0.05 on a unit mesh: the parabola's face deviations (-0.38125,
    # +0.14375) exceed 2 * 0.05 * 0.5 = 0.05 and are cut to it
    qm, qp, shaped = oracle.parabola(0.0, 1.0, 1.05, 0.0, 1.0, 2.0, 0.5, 1.5)
    assert shaped
    assert qp == pytest.approx(1.05, rel=1e-15) and qm == pytest.approx(0.95, rel=1e-15)
    # a gentle curvature is kept: slopes 1 and 0.8 give a = -0.1, b = 0.9 and face
    # deviations -0.475 / +0.425, inside the bounds -0.8 / +0.8
    qm, qp, _ = oracle.parabola(0.0, 1.0, 1.8, 0.0, 1.0, 2.0, 0.5, 1.5)
    assert qm == pytest.approx(0.525, rel=1e-14) and qp == pytest.approx(1.425, rel=1e-14)


def test_limiter_is_lipschitz():
    """No branch of the limiter jumps: a perturbation of the data by d moves the
    face values by at most a few d (continuity keeps nearby runs nearby)."""
    rng = np.random.default_rng(3)
    xc, xf = _log_mesh(60)
    for _ in range(4000):
        i = int(rng.integers(1, 58))
        v = rng.normal(size=3)
        v[1] = v[0] + rng.choice([-1, 1]) * rng.uniform(0, 1e-6) if rng.uniform() < 0.2 else v[1]
        d = 1e-9 * rng.normal(size=3)
        args = (xc[i - 1], xc[i], xc[i + 1], xf[i], xf[i + 1])
        q1 = oracle.parabola(*v, *args)
        q2 = oracle.parabola(*(v + d), *args)
        bound = 8 * np.abs(d).max() * (1 + (xc[i + 1] - xc[i - 1]) / min(xc[i] - xc[i - 1], xc[i + 1] - xc[i]))
        assert abs(q2[0] - q1[0]) <= bound and abs(q2[1] - q1[1]) <= bound


def test_no_new_extrema_random():
    rng = np.random.default_rng(7)
    xc, xf = _log_mesh(200)
    for _ in range(20):
        v = np.cumsum(rng.normal(size=xc.size)) + rng.normal(size=xc.size) * rng.uniform(0, 3)
        for i in range(1, xc.size - 1):
            qm, qp, _ = oracle.parabola(v[i - 1], v[i], v[i + 1], xc[i - 1], xc[i], xc[i + 1], xf[i], xf[i + 1])
            assert min(v[i - 1], v[i]) - 1e-14 <= qm <= max(v[i - 1], v[i]) + 1e-14
            assert min(v[i], v[i + 1]) - 1e-14 <= qp <= max(v[i], v[i + 1]) + 1e-14


@pytest.fixture(scope="module")
def disc_oracle():
    return oracle.Oracle(syn.scaled(syn.DISC_NOISE, 8, 4, 32, steps=1))


@pytest.mark.parametrize("r,z", [(0.6, 0.0), (0.6, 0.03), (1.0, 0.1), (1.7, -0.12), (1.3, 0.05)])
def test_hydrostatic_and_centrifugal_balance(disc_oracle, r, z):
    o = disc_oracle
    gm = o.w.gm
    rho, vth, p = o.eq_prim(r, z)
    R3 = (r * r + z * z) ** 1.5
    h = 1e-5
    dpdz = (o.eq_prim(r, z + h)[2] - o.eq_prim(r, z - h)[2]) / (2 * h)
    assert dpdz == pytest.approx(-gm * z * rho / R3, rel=1e-7, abs=1e-9 * p / 0.05)
    dpdr = (o.eq_prim(r + h, z)[2] - o.eq_prim(r - h, z)[2]) / (2 * h)
    assert dpdr == pytest.approx(rho * (vth * vth / r - gm * r / R3), rel=1e-7)


@pytest.mark.parametrize("r", [0.6, 1.0, 1.8])
def test_column_mass_is_surface_density(disc_oracle, r):
    o = disc_oracle
    sigma0, beta_sigma, T0, beta_T = o.w.disc
    H = math.sqrt(2.0 * T0 * r ** beta_T) / math.sqrt(o.w.gm / r ** 3)
    z = np.linspace(-12 * H, 12 * H, 40001)
    rho = np.array([o.eq_prim(r, zz)[0] for zz in z])
    sigma = np.trapezoid(rho, z)
    h2 = (H / r) ** 2
    assert sigma == pytest.approx(sigma0 * r ** beta_sigma, rel=3 * h2)


def test_frame_velocity(disc_oracle):
    o = disc_oracle
    E0 = o.equilibrium_state()
    rc, _ = o.coords(0)
    zc, _ = o.coords(2)
    k, i = 7, 3
    rho, vth, p = o.eq_prim(rc[i], zc[k])
    assert E0[syn.F_MV, k, 0, i] / E0[syn.F_RHO, k, 0, i] == pytest.approx(vth - o.w.omega_frame * rc[i], rel=1e-14)
    P = (o.w.gamma - 1) * (E0[syn.F_EN] - 0.5 * E0[syn.F_MV] ** 2 / E0[syn.F_RHO])
    assert P[k, 0, i] == pytest.approx(p, rel=1e-12)
