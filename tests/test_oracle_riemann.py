"""Pins of the oracle's exact Riemann solver (Sect. 2.6, Toro ch. 4).

The solver is checked against relations it does not itself evaluate: the
Rankine-Hugoniot jump conditions across each shock, isentropy and the Riemann
invariant across each rarefaction, conservation of the whole self-similar
solution (integrated numerically), Galilean invariance, and exact return of
the state for identical left/right data.  Cases are chosen to cover every wave
pattern: rarefaction-shock (the Sod problem of the Box workload),
rarefaction-rarefaction, shock-shock, shock-rarefaction, a transonic fan, a
supersonic flow and vacuum generation.
"""
import numpy as np
import pytest

import oracle

G = 1.4
CASES = {
    "sod": ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1)),
    "rar_rar": ((1.0, -1.0, 1.0), (1.0, 1.0, 1.0)),
    "shock_shock": ((1.0, 2.0, 1.0), (1.0, -2.0, 1.0)),
    "rar_shock_strong": ((1.0, 0.0, 100.0), (1.0, 0.0, 0.01)),
    "shock_rar_strong": ((1.0, 0.0, 0.01), (1.0, 0.0, 100.0)),
    "transonic_fan": ((1.0, 0.5, 1.0), (0.125, 0.5, 0.1)),
    "supersonic": ((1.0, 3.0, 1.0), (0.5, 3.0, 0.5)),
    "asymmetric": ((2.0, 0.3, 3.0), (0.7, -0.4, 0.5)),
}


def _cons(W):
    rho, u, p = W
    return np.array([rho, rho * u, 0.5 * rho * u * u + p / (G - 1.0)])


def _flux(W):
    rho, u, p = W
    E = 0.5 * rho * u * u + p / (G - 1.0)
    return np.array([rho * u, rho * u * u + p, (E + p) * u])


def _c(W):
    return np.sqrt(G * W[2] / W[0])


@pytest.mark.parametrize("name", sorted(CASES))
def test_wave_relations(name):
    WL, WR = CASES[name]
    _, ps, us, iters, conv, _, vac = oracle.riemann(G, WL, WR)
    assert conv and not vac
    eps = 1e-7 * max(1.0, abs(us))
    starL, *_ = oracle.riemann(G, WL, WR, S=us - eps)
    starR, *_ = oracle.riemann(G, WL, WR, S=us + eps)
    assert starL[2] == pytest.approx(ps, rel=1e-12) and starR[2] == pytest.approx(ps, rel=1e-12)
    assert starL[1] == pytest.approx(us, rel=1e-12, abs=1e-12)
    for W, star, sgn in ((WL, starL, -1), (WR, starR, +1)):
        if ps > W[2]:  # shock: Rankine-Hugoniot with the speed from mass conservation
            S = (star[0] * star[1] - W[0] * W[1]) / (star[0] - W[0])
            jump = (_flux(star) - S * _cons(star)) - (_flux(W) - S * _cons(W))
            scale = np.abs(_flux(W) - S * _cons(W)) + np.abs(_flux(star)) + np.abs(S * _cons(star))
            assert np.all(np.abs(jump) <= 1e-11 * scale), (name, sgn, jump)
            assert (S - W[1]) * sgn > 0  # shock moves away from the contact into the data
        else:  # rarefaction: isentropic and the Riemann invariant across the fan is constant
            assert star[2] / star[0] ** G == pytest.approx(W[2] / W[0] ** G, rel=1e-11)
            inv_data = W[1] - sgn * 2.0 * _c(W) / (G - 1.0)
            inv_star = star[1] - sgn * 2.0 * _c(star) / (G - 1.0)
            assert inv_star == pytest.approx(inv_data, rel=1e-11, abs=1e-11)


@pytest.mark.parametrize("name", sorted(CASES) + ["vacuum"])
def test_global_conservation(name):
    """The self-similar solution at t = 1 conserves mass, momentum and energy:
    int_{-X}^{X} U dx = X (U_L + U_R) + F(U_L) - F(U_R)."""
    WL, WR = CASES.get(name, ((1.0, -4.0, 0.4), (1.0, 4.0, 0.4)))
    X = 60.0
    S = np.linspace(-X, X, 120001)
    U = np.array([_cons(oracle.riemann(G, WL, WR, S=s)[0]) for s in S])
    integral = np.trapezoid(U, S, axis=0)
    expect = X * (_cons(WL) + _cons(WR)) + _flux(WL) - _flux(WR)
    # the trapezoid rule errs by at most dS/2 times each jump of a piecewise-smooth integrand
    dS = S[1] - S[0]
    bound = dS * np.abs(np.diff(U, axis=0)).sum(axis=0) + 1e-9 * (np.abs(expect) + 1.0)
    assert np.all(np.abs(integral - expect) <= bound), (name, integral, expect, bound)


def test_vacuum_generation():
    WL, WR = (1.0, -4.0, 0.4), (1.0, 4.0, 0.4)
    W, ps, us, _, _, side, vac = oracle.riemann(G, WL, WR)
    assert vac and side == 0 and W[0] == 0.0 and W[2] == 0.0
    # left fan edge speeds: head u_L - c_L, vacuum front u_L + 2 c_L/(gamma-1)
    cl = _c(WL)
    front = WL[1] + 2.0 * cl / (G - 1.0)
    Wf, *_ = oracle.riemann(G, WL, WR, S=0.5 * (WL[1] - cl + front))
    assert Wf[1] + 2.0 * _c(Wf) / (G - 1.0) == pytest.approx(WL[1] + 2.0 * cl / (G - 1.0), rel=1e-12)


@pytest.mark.parametrize("u", [0.0, 0.3, 2.5, -2.5, -0.7])
def test_identical_states_exact(u):
    W0 = (0.7, u, 0.3)
    for S in (0.0, 0.1, -0.1):
        W, ps, us, _, conv, _, _ = oracle.riemann(G, W0, W0, S=S)
        assert conv and ps == W0[2] and us == u
        assert tuple(W) == W0


@pytest.mark.parametrize("name", ["sod", "asymmetric", "shock_shock"])
def test_galilean_invariance(name):
    WL, WR = CASES[name]
    U = 0.37
    _, ps, us, *_ = oracle.riemann(G, WL, WR)
    sl = (WL[0], WL[1] + U, WL[2])
    sr = (WR[0], WR[1] + U, WR[2])
    _, ps2, us2, *_ = oracle.riemann(G, sl, sr)
    assert ps2 == pytest.approx(ps, rel=1e-12)
    assert us2 == pytest.approx(us + U, rel=1e-12)
    for S in (-0.8, -0.1, 0.2, 0.9):
        W1, *_ = oracle.riemann(G, WL, WR, S=S)
        W2, *_ = oracle.riemann(G, sl, sr, S=S + U)
        assert W2[0] == pytest.approx(W1[0], rel=1e-11)
        assert W2[1] == pytest.approx(W1[1] + U, rel=1e-11, abs=1e-12)
        assert W2[2] == pytest.approx(W1[2], rel=1e-11)


def test_mirror_symmetry():
    WL, WR = CASES["asymmetric"]
    mL = (WR[0], -WR[1], WR[2])
    mR = (WL[0], -WL[1], WL[2])
    for S in (-1.2, -0.3, 0.0, 0.4, 1.1):
        W1, *_ = oracle.riemann(G, WL, WR, S=S)
        W2, *_ = oracle.riemann(G, mL, mR, S=-S)
        assert W2[0] == pytest.approx(W1[0], rel=1e-11)
        assert W2[1] == pytest.approx(-W1[1], rel=1e-11, abs=1e-12)
        assert W2[2] == pytest.approx(W1[2], rel=1e-11)
