"""Symmetry pins of the oracle's step on the disc (Sects. 2.2-2.5).

The scheme treats every azimuthal cell alike and the disc is symmetric about
its midplane, so:
- rolling a non-axisymmetric state (the jittered bi-fluid vortex) by whole
  cells in theta rolls the step result, bit for bit (a wrong periodic wrap or
  ghost index in theta breaks it);
- mirroring the state about z = 0 (with w -> -w for gas and dust) mirrors the
  result, to rounding (the two faces of a cell are summed in the opposite
  order); a z-face, z-ghost or z-coordinate index that is not symmetric breaks
  it (the signs of the vertical forces are pinned against the potential in
  test_oracle_sources.py: a flipped one would still be odd in z).
"""
import numpy as np
import pytest

import oracle
import synthetic as syn
from tests.parity import jitter

MU, MV, MW, EN, RHO, DMU, DMV, DMW, DRHO = range(9)


def _state():
    w = syn.scaled(syn.VORTEX, 12, 10, 32)
    o = oracle.Oracle(w)
    E = jitter(oracle.initial_state(o), w.gamma, np.random.default_rng(9), 1e-3)
    return w, o, E


@pytest.mark.parametrize("shift", [1, 3, 7])
def test_theta_translation_is_exact(shift):
    w, o, E = _state()
    dt = o.cfl_dt(E)
    a = np.roll(o.step(E, dt), shift, axis=2)
    b = o.step(np.roll(E, shift, axis=2), dt)
    assert o.take_status() == 0
    assert np.array_equal(a, b)


def _mirror(E):
    M = E[:, ::-1].copy()
    M[MW] *= -1.0
    M[DMW] *= -1.0
    return M


def test_midplane_mirror():
    w, o, E = _state()
    dt = o.cfl_dt(E)
    a = _mirror(o.step(E, dt))
    b = o.step(_mirror(E), dt)
    assert o.take_status() == 0
    scale = np.abs(a).max(axis=(1, 2, 3), keepdims=True)
    assert (np.abs(a - b) / scale).max() <= 1e-12
    # and the vertical momentum really moved (the check is not vacuous)
    assert np.abs(a[MW] - _mirror(E)[MW]).max() > 1e-6 * scale[MW].max()
