"""The linear RWI growth rates the RWI runs are held to (Sect. 4.3), on the
oracle's midplane equilibrium.

Checks of the eigenvalue solver itself: the unbumped Keplerian disc has no
growing mode at r0 (it is linearly stable: no RWI without an extremum of the
vortensity-entropy function); a barotropic bump (P = K rho^Gamma), the textbook
RWI case, grows with its corotation at the bump, faster for a taller bump; the
rates converge under mesh refinement.  Then the two statements the RWI
workload rests on: a bump as wide as H(r0) gives no growing mode in this disc,
and the workload's bump (delta = 0.5, Delta_r = H(r0) / 2) grows at rates of
order 0.1 Omega(r0), rising with m from 2 to 6.
"""
from dataclasses import replace
import math

import numpy as np

import oracle
import synthetic as syn
from tests.rwi_linear import rwi_growth_rate, rwi_modes

R_IN, R_OUT = 0.6, 1.6


def _background(delta, width):
    o = oracle.Oracle(replace(syn.scaled(syn.RWI, 8, 4, 4), rwi_delta=delta, rwi_width=width))
    return lambda r: o.eq_prim(r, 0.0)


def _barotropic(amp, width, cs=0.1, gamma=5.0 / 3.0):
    """rho = 1 + (A - 1) exp(-(r - 1)^2 / (2 width^2)), P = K rho^gamma with
    sound speed cs at the base, Omega from radial balance about GM = 1."""
    K = cs * cs / gamma

    def bg(r):
        def rho(x):
            return 1.0 + (amp - 1.0) * math.exp(-(x - 1.0) ** 2 / (2.0 * width * width))
        h = 1e-6
        dP = K * (rho(r + h) ** gamma - rho(r - h) ** gamma) / (2.0 * h)
        return rho(r), math.sqrt(1.0 / r + r * dP / rho(r)), K * rho(r) ** gamma
    return bg


def test_keplerian_disc_without_bump_has_no_growing_mode():
    bg = _background(0.0, 0.025)
    for m in (2, 4, 6):
        assert rwi_growth_rate(bg, m, 1.0, R_IN, R_OUT, n=200) < 1e-3


def test_barotropic_bump_grows_at_corotation():
    rates = []
    for amp in (1.25, 1.5):
        bg = _barotropic(amp, 0.05)
        ev = rwi_modes(bg, 4, 0.5, R_OUT, n=200, gamma=5.0 / 3.0)
        top = ev[0]
        om0 = bg(1.0)[1]
        assert abs(top.real / (4 * om0) - 1.0) < 0.05, top   # corotation at the bump
        rates.append(top.imag)
    assert 0.05 < rates[0] < rates[1] < 1.0, rates


def test_rates_converge_under_refinement():
    bg = _background(0.5, 0.025)
    a, b = rwi_growth_rate(bg, 4, 1.0, R_IN, R_OUT, n=200), rwi_growth_rate(bg, 4, 1.0, R_IN, R_OUT, n=400)
    assert a > 0.05 and abs(a - b) <= 0.01 * b, (a, b)


def test_bump_as_wide_as_H_is_stable():
    for delta in (0.5, 1.0):
        bg = _background(delta, 0.05)
        assert rwi_growth_rate(bg, 4, 1.0, R_IN, R_OUT, n=200) < 1e-3, delta


def test_workload_bump_grows():
    w = syn.RWI
    bg = _background(w.rwi_delta, w.rwi_width)
    rates = [rwi_growth_rate(bg, m, w.rwi_r0, R_IN, R_OUT, n=200) for m in (2, 4, 6)]
    print("linear growth rates m = 2, 4, 6:", [f"{g:.4f}" for g in rates])
    assert 0.04 < rates[0] < rates[1] < rates[2] < 0.2, rates
    assert np.isclose(rates[1], 0.111, atol=0.003), rates
