"""Drag law 2 (Epstein with the Stokes regime of Sect. 2.9, reading R19) on the
GPU against the oracle: the bi-fluid vortex with kappa chosen so that the
switch splits the disc, 15 steps on the oracle's dt sequence (the oracle's
own drift from a 1e-15 input perturbation is 4e-13 after 15 steps), FP64 and the FP64
perturbation form <= 1e-12, FP32 <= 1e-5; the regime moves the dust far more
than the bar; the adjoint refuses the law."""
from dataclasses import replace

import numpy as np
import pytest

import oracle
import synthetic as syn
from tests.parity import rel_l1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2207_04252_gb300 import build
    build.build()
    from paper_2207_04252_gb300 import rossbi, workloads
    torch.cuda.init()
    return rossbi, workloads


@pytest.fixture(scope="module")
def reference():
    base = replace(syn.scaled(syn.VORTEX, 20, 18, 32), drag_law=1)
    o1 = oracle.Oracle(base)
    E0 = oracle.initial_state(o1)
    kappa = 2.25 / float(np.median(E0[4]))
    w = replace(base, drag_law=2, drag_kappa=kappa)
    o = oracle.Oracle(w)
    E, _, dts = o.run(E0.copy(), steps=15)
    assert o.take_status() == 0
    E1, _, _ = o1.run(E0.copy(), dts=dts)
    return w, o, E, E1, dts


@pytest.mark.parametrize("form", ["fp64", "fp64_pert", "fp32_pert"])
def test_stokes_regime_parity(lib, reference, form):
    R, W = lib
    w, o, E_ref, E_law1, dts = reference
    prec = {"fp64": R.ROSSBI_FP64, "fp64_pert": R.ROSSBI_FP64_PERT, "fp32_pert": R.ROSSBI_FP32_PERT}[form]
    tol = 1e-5 if form == "fp32_pert" else 1e-12
    g = W.Grid(w, precision=prec)
    s = g.initial_state("cuda")
    for dt in dts:
        g.step(s, dt=dt)
    assert g.take_status() == 0
    errs = rel_l1(g.full_state(s), E_ref, o.volumes())
    assert all(e <= tol for e in errs.values()), errs
    off = rel_l1(E_law1, E_ref, o.volumes())
    assert off["dust_momentum"] > 100 * max(tol, errs["dust_momentum"]), (off, errs)
    g.close()


def test_adjoint_refuses_the_stokes_regime(lib, reference):
    import torch
    R, W = lib
    w = reference[0]
    g = W.Grid(w)
    s = g.initial_state("cuda")
    with pytest.raises(R.RossbiError) as e:
        g.adjoint_step(s, 1e-3, torch.ones_like(s))
    assert e.value.code == R.ROSSBI_ERR_UNSUPPORTED
    g.close()
