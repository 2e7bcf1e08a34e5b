"""Pins of the oracle's indirect-gravity term (Sect. 2.10, reading R16).

The paper gives the gradient of the indirect potential in cylindrical
components, X_ref (A cos(theta) + B sin(theta), -A sin(theta) + B cos(theta), 0),
with A and B moments of the disc mass.  The physics behind it: the disc pulls
the star with the acceleration a = G sum_j m_j x_j / |x_j|^3 (Cartesian
positions x_j of the masses relative to the star), and in the star's frame
every parcel of gas and dust feels -a.  The pins below check the oracle's
cylindrical formula against that Cartesian brute force, and against the
symmetries it must have: an axisymmetric disc exerts no pull, and turning the
disc by whole cells in theta turns the force with it.
"""
import numpy as np
import pytest

import oracle
import synthetic as syn
from tests.parity import jitter

MU, MV, MW, EN, RHO, DMU, DMV, DMW, DRHO = range(9)  # field order of App. B


def _grid(o):
    r, _ = o.coords(0)
    th, _ = o.coords(1)
    z, _ = o.coords(2)
    Z, TH, R = np.meshgrid(z, th, r, indexing="ij")  # (nz, nth, nr)
    return R, TH, Z, o.volumes()[None, None, :]


def bump(E, r, th, z, amp=0.05, th0=1.0, width=0.6):
    """An m = 1 asymmetry of the disc mass: every gas field scaled by
    1 + amp exp(-(dtheta/width)^2 - ((r - 1.1)/0.25)^2 - (z/0.08)^2) about
    theta = th0 and, with dust, every dust field likewise about th0 + 2
    (velocities and temperature unchanged, so the bump is a mild density and
    pressure excess, away from the domain's edges and symmetric in z).
    r, th, z: cell-centre coordinates; E: full conservative state
    (nf, nz, nth, nr)."""
    E = E.copy()
    win = np.exp(-((r[None, None, :] - 1.1) / 0.25) ** 2 - (z[:, None, None] / 0.08) ** 2)
    groups = ((slice(0, 5), th0), (slice(5, 9), th0 + 2.0))
    for fs, c in groups[:1 if E.shape[0] == 5 else 2]:
        dth = np.angle(np.exp(1j * (th[None, :, None] - c)))
        E[fs] *= (1.0 + amp * win * np.exp(-(dth / width) ** 2))[None]
    return E


def _lopsided(o):
    return bump(oracle.initial_state(o), o.coords(0)[0], o.coords(1)[0], o.coords(2)[0])


def _indirect_part(o, E, x_ref):
    """G(E) with the indirect term minus G(E) without it."""
    o.set_indirect(x_ref)
    g_on = o.rhs(E)
    o.set_indirect(0.0)
    g_off = o.rhs(E)
    assert o.take_status() == 0
    return g_on - g_off


def _cartesian_brute_force(o, E, x_ref):
    """The indirect source of every cell from the star's Cartesian
    acceleration: full gas plus dust mass, point masses at cell centres."""
    R, TH, Z, V = _grid(o)
    X, Y = R * np.cos(TH), R * np.sin(TH)
    m = V * (E[RHO] + (E[DRHO] if o.nf > 5 else 0.0))
    d3 = (X * X + Y * Y + Z * Z) ** 1.5
    a = x_ref * np.array([(m * X / d3).sum(), (m * Y / d3).sum()])  # z dropped, as in the paper
    # force per unit mass on the fluid, -a, in the local (r, theta) basis
    fr = -(a[0] * np.cos(TH) + a[1] * np.sin(TH))
    ft = -(-a[0] * np.sin(TH) + a[1] * np.cos(TH))
    D = np.zeros_like(E)
    D[MU] = V * E[RHO] * fr
    D[MV] = V * E[RHO] * ft
    D[EN] = V * (E[MU] * fr + E[MV] * ft)
    if o.nf > 5:
        D[DMU] = V * E[DRHO] * fr
        D[DMV] = V * E[DRHO] * ft
    return D, a


@pytest.mark.parametrize("dust", [True, False])
def test_indirect_matches_cartesian_newtonian_pull(dust):
    w = syn.scaled(syn.VORTEX if dust else syn.DISC_NOISE, 16, 12, 16)
    o = oracle.Oracle(w)
    E = _lopsided(o)
    D = _indirect_part(o, E, 0.7)
    ref, a = _cartesian_brute_force(o, E, 0.7)
    assert np.hypot(*a) > 1e-3  # the pull is not negligible
    for f in range(o.nf):
        scale = np.abs(ref[f]).max()
        if f in (MW, RHO, DMW, DRHO):
            assert not D[f].any(), f
            continue
        assert np.abs(D[f] - ref[f]).max() <= 1e-10 * scale, (f, np.abs(D[f] - ref[f]).max() / scale)
    # A and B as the oracle reports them are the brute-force pull (and vanish when off)
    assert not o.indirect(E).any()
    o.set_indirect(0.7)
    assert np.allclose(o.indirect(E), a, rtol=1e-10, atol=0)


def test_axisymmetric_disc_exerts_no_pull():
    w = syn.scaled(syn.VORTEX, 16, 12, 16)
    o = oracle.Oracle(w)
    E = o.equilibrium_state()
    R, TH, Z, _ = _grid(o)
    E[RHO] *= 1.0 + 0.05 * np.exp(-((R - 1.1) / 0.2) ** 2)  # a ring: m = 0
    E[DRHO] = 0.01 * E[RHO]
    D = _indirect_part(o, E, 0.7)
    lop = _indirect_part(o, _lopsided(o), 0.7)
    for f in (MU, MV, EN, DMU, DMV):
        assert np.abs(D[f]).max() <= 1e-12 * np.abs(lop[f]).max(), f


@pytest.mark.parametrize("shift", [1, 5])
def test_turning_the_disc_turns_the_force(shift):
    """Rolling every field by whole cells in theta rolls the indirect source
    with it: its local (r, theta) components are those of a rotated vector.
    A sign or a cos/sin swap in the cylindrical formula breaks this."""
    w = syn.scaled(syn.VORTEX, 16, 12, 16)
    o = oracle.Oracle(w)
    E = _lopsided(o)
    D = _indirect_part(o, E, 0.7)
    Dr = _indirect_part(o, np.roll(E, shift, axis=2), 0.7)
    scale = np.abs(D).max(axis=(1, 2, 3), keepdims=True) + 1e-300
    assert (np.abs(Dr - np.roll(D, shift, axis=2)) / scale).max() <= 1e-12


def test_equilibrium_stays_bit_exact_with_indirect_gravity():
    w = syn.scaled(syn.DISC_NOISE, 16, 12, 16)
    o = oracle.Oracle(w)
    o.set_indirect(1.0)
    E = o.equilibrium_state()
    assert not o.indirect(E).any()
    dt = o.cfl_dt(E)
    assert np.array_equal(o.step(o.step(E, dt), dt), E)


def test_box_has_no_indirect_term():
    w = syn.scaled(syn.SOD, 16, 2, 2)
    o = oracle.Oracle(w)
    o.set_indirect(1.0)
    E = oracle.initial_state(o)
    assert not o.indirect(E).any()
    with_term = o.step(E, 1e-3)
    o.set_indirect(0.0)
    assert np.array_equal(with_term, o.step(E, 1e-3))


def test_sampled_steps_refuse_the_global_term():
    w = syn.scaled(syn.VORTEX, 16, 12, 16)
    o = oracle.Oracle(w)
    o.set_indirect(1.0)
    E = oracle.initial_state(o)
    with pytest.raises(ValueError):
        o.step_sampled(E, 1e-3, [0, 1])


def test_tlm_carries_the_indirect_term():
    """Tangent-linear step with the global A, B against central differences
    of the step, along a density direction that moves A and B."""
    w = syn.scaled(syn.VORTEX, 16, 12, 32)
    o = oracle.Oracle(w)
    o.set_indirect(0.7)
    rng = np.random.default_rng(5)
    E = jitter(_lopsided(o), w.gamma, rng, 1e-3)
    R, TH, Z, _ = _grid(o)
    # smooth m = 1 density directions that move A and B; momenta and gas
    # energy scale with the densities, so no velocity moves (a moving dust
    # velocity would flip the upwind branch at corotation, where v_d = 0)
    d = np.zeros_like(E)
    d[RHO] = 1e-2 * E[RHO] * np.cos(TH - 0.3)
    d[DRHO] = 1e-2 * E[DRHO] * np.sin(TH)
    for f in (MU, MV, MW, EN):
        d[f] = E[f] / E[RHO] * d[RHO]
    for f in (DMU, DMV, DMW):
        d[f] = E[f] / E[DRHO] * d[DRHO]
    dt = o.cfl_dt(E)
    _, t = o.step_tlm(E, d, dt)
    assert o.take_status() == 0
    o.set_indirect(0.0)
    _, t0 = o.step_tlm(E, d, dt)
    o.set_indirect(0.7)

    def central(h):
        return (o.step(E + h * d, dt) - o.step(E - h * d, dt)) / (2 * h)

    num = np.abs(t - t0).sum(axis=(1, 2, 3))
    assert num[[MU, MV, DMU, DMV]].min() > 0  # the indirect term moves the tangent
    err = min((np.abs(central(h) - t).sum(axis=(1, 2, 3)) / np.abs(t).sum(axis=(1, 2, 3))
               for h in (1e-5, 3e-6)), key=lambda e: e.max())
    assert err.max() <= 1e-6, err
