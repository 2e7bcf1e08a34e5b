"""Pins of the oracle's several dust species (reading R20; Sect. 5.4 names the
multi-fluid approach).

The species are independent pressureless fluids, each coupled to the gas only
by its own drag, so:
- splitting one dust fluid into two identical species of half its density
  changes nothing: the gas evolves as before and the species add up to the
  single fluid (halving is exact in binary; the drag's closed forms for one
  and for several species differ only by rounding);
- a second species of zero density leaves the single-species step unchanged;
- the multi-species drag is the backward-Euler solution of the coupled
  relaxation, here solved independently as a linear system with numpy, and it
  conserves the total momentum;
- the tangent-linear step agrees with central differences.
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle
import synthetic as syn
from tests.parity import jitter


def _w(nd, **kw):
    return replace(syn.scaled(syn.VORTEX, 12, 10, 16), n_dust=nd, **kw)


def _scale(A):
    """Per-field scale for comparisons: a momentum component is measured
    against the whole momentum vector (the small radial and vertical
    components carry the rounding of the large azimuthal one, as in the
    parity measure, reading R13)."""
    m = np.abs(A).max(axis=(1, 2, 3))
    groups = [(0, 1, 2), (3,), (4,)] + [tuple(range(5 + 4 * s, 8 + 4 * s)) for s in range((len(m) - 5) // 4)] + \
             [(8 + 4 * s,) for s in range((len(m) - 5) // 4)]
    out = np.empty_like(m)
    for g in groups:
        out[list(g)] = m[list(g)].max()
    return out[:, None, None, None]


def _one_and_two():
    o1, o2 = oracle.Oracle(_w(1)), oracle.Oracle(_w(2))
    E1 = jitter(oracle.initial_state(o1), o1.w.gamma, np.random.default_rng(4), 1e-3)
    E2 = np.zeros((13,) + E1.shape[1:])
    E2[:5] = E1[:5]
    E2[5:9] = 0.5 * E1[5:9]
    E2[9:13] = 0.5 * E1[5:9]
    return o1, o2, E1, E2


def test_two_half_species_are_one():
    o1, o2, E1, E2 = _one_and_two()
    dt = o1.cfl_dt(E1)
    assert o2.cfl_dt(E2) == dt
    A, B = o1.step(E1, dt), o2.step(E2, dt)
    assert o1.take_status() == 0 and o2.take_status() == 0
    scale = _scale(A)
    assert (np.abs(B[:5] - A[:5]) / scale[:5]).max() <= 1e-13
    assert np.array_equal(B[5:9], B[9:13])                       # the two halves stay twins
    assert (np.abs(B[5:9] + B[9:13] - A[5:9]) / scale[5:9]).max() <= 1e-13


def test_an_empty_second_species_changes_nothing():
    o1, o2, E1, E2 = _one_and_two()
    E2[5:9] = E1[5:9]
    E2[9:13] = 0.0
    dt = o1.cfl_dt(E1)
    A, B = o1.step(E1, dt), o2.step(E2, dt)
    scale = _scale(A)
    assert (np.abs(B[:9] - A) / scale).max() <= 1e-13
    assert not B[9:13].any()


def test_multispecies_drag_is_the_backward_euler_solution():
    """One cell, three species with different Stokes numbers: the oracle's
    closed form against numpy's solution of the linear backward-Euler system,
    per velocity component; total momentum conserved."""
    w = replace(syn.scaled(syn.VORTEX, 12, 10, 16), n_dust=3)
    o = oracle.Oracle(w)
    f = np.array([1.0, 0.3, 4.0])
    o.set_species_stokes(f)
    rng = np.random.default_rng(5)
    rg, P = 1.3, 0.02
    vg = rng.uniform(-0.2, 0.2, 3)
    U = np.zeros(17)
    U[4], U[0:3], U[3] = rg, rg * vg, P / 0.4 + 0.5 * rg * vg @ vg
    rd = np.array([0.02, 0.05, 0.01])
    vd = rng.uniform(-0.2, 0.2, (3, 3))
    for s in range(3):
        U[5 + 4 * s + 3] = rd[s]
        U[5 + 4 * s:8 + 4 * s] = rd[s] * vd[s]
    i, tau = 4, 0.05
    out = o.drag(i, U, tau)
    r = o.coords(0)[0][i]
    ts = w.stokes * f / np.sqrt(w.gm / r ** 3)       # constant-St law: t_k = St_k / Omega_K(r)
    a = tau / ts
    for c in range(3):
        # unknowns (v_g, v_1, v_2, v_3): rho_g (v_g - vg) = sum rho_k a_k (v_k - v_g),
        # v_k - vd_k = -a_k (v_k - v_g)
        M = np.zeros((4, 4))
        rhs = np.zeros(4)
        M[0, 0] = rg + (rd * a).sum()
        M[0, 1:] = -rd * a
        rhs[0] = rg * vg[c]
        for s in range(3):
            M[1 + s, 1 + s] = 1.0 + a[s]
            M[1 + s, 0] = -a[s]
            rhs[1 + s] = vd[s, c]
        v = np.linalg.solve(M, rhs)
        assert out[c] / rg == pytest.approx(v[0], rel=1e-12, abs=1e-15)
        for s in range(3):
            assert out[5 + 4 * s + c] / rd[s] == pytest.approx(v[1 + s], rel=1e-12, abs=1e-15)
        tot0 = U[c] + sum(U[5 + 4 * s + c] for s in range(3))
        tot1 = out[c] + sum(out[5 + 4 * s + c] for s in range(3))
        assert tot1 == pytest.approx(tot0, rel=1e-14, abs=1e-16)


def test_tlm_with_two_species():
    w = _w(2)
    o = oracle.Oracle(w)
    o.set_species_stokes([1.0, 0.25])
    rng = np.random.default_rng(6)
    E = jitter(oracle.initial_state(o), w.gamma, rng, 1e-3)
    dt = o.cfl_dt(E)
    for f, (k, j, i) in ((12, (8, 4, 6)), (10, (7, 3, 5)), (4, (9, 5, 7))):
        d = np.zeros_like(E)
        d[f, k, j, i] = 1e-3 * abs(E[f, k, j, i]) + 1e-12
        _, t = o.step_tlm(E, d, dt)
        err = min(np.abs((o.step(E + h * d, dt) - o.step(E - h * d, dt)) / (2 * h) - t).max()
                  for h in (1e-3, 1e-4, 1e-5, 1e-6))
        assert err <= 1e-4 * np.abs(t).max(), (f, err / np.abs(t).max())
    assert o.take_status() == 0
