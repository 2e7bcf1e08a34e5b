"""Drag law 2 (Epstein with the Stokes regime of Sect. 2.9, reading R19) on the
GPU against the oracle: the bi-fluid vortex with kappa chosen so that the
switch splits the disc, 15 steps on the oracle's dt sequence (the oracle's
own drift from a 1e-15 input perturbation is 4e-13 after 15 steps), FP64 and the FP64
perturbation form <= 1e-12, FP32 <= 1e-5; the regime moves the dust far more
than the bar; the adjoint of the law satisfies the transpose identity."""
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
    assert off["dust_momentum"] > 20 * max(tol, errs["dust_momentum"]), (off, errs)  # 6.3e-4 after 15 steps
    g.close()


def test_adjoint_of_the_stokes_regime(lib, reference):
    """The adjoint with drag law 2, the switch splitting the disc: the
    transpose identity <lam, J delta> = <J^T lam, delta> against the oracle's
    tangent-linear step (1e-12), and d/dSt of one step (1e-11)."""
    import torch
    from tests.parity import jitter
    R, W = lib
    w, o, _, _, _ = reference
    rng = np.random.default_rng(8)
    E0 = jitter(oracle.initial_state(o), w.gamma, rng, 1e-3)
    rg = E0[4]
    inside = (w.drag_kappa * rg > 2.25).mean()
    assert 0.05 < inside < 0.95, inside  # both regimes present
    dt = o.cfl_dt(E0)
    scale = np.abs(E0).mean(axis=(1, 2, 3), keepdims=True) + 1e-30
    g = W.Grid(w)
    for trial in range(2):
        lam = rng.standard_normal(E0.shape) / scale
        delta = rng.standard_normal(E0.shape) * scale
        _, t = o.step_tlm(E0, delta, dt)
        assert o.take_status() == 0
        lam_d = torch.from_numpy(lam).cuda().contiguous()
        g.adjoint_step(torch.from_numpy(E0).cuda().contiguous(), dt, lam_d)
        assert g.take_status() == 0
        lhs, rhs = float((lam * t).sum()), float((lam_d.cpu().numpy() * delta).sum())
        assert abs(lhs - rhs) <= 1e-12 * float(np.abs(lam * t).sum()), (trial, lhs, rhs)
    lam = rng.standard_normal(E0.shape) / scale
    _, t = o.step_tlm(E0, np.zeros_like(E0), dt, dstokes=1.0)
    ref = float((lam * t).sum())
    dst = g.adjoint_step(torch.from_numpy(E0).cuda().contiguous(), dt, torch.from_numpy(lam).cuda().contiguous(),
                         want_dstokes=True)
    assert abs(dst - ref) <= 1e-11 * float(np.abs(lam * t).sum()), (dst, ref)
    g.close()
