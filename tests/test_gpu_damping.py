"""The wave-killing zones (Sect. 2.4, reading R17) on the GPU against the oracle.

Runs follow the oracle's dt sequence with the zones on (edges 1.25 r_in and
0.84 r_out, tau a hundredth of the boundary's orbital period, so the term is
far above the parity bars): FP64 and the FP64 perturbation form <= 1e-12,
FP32 <= 1e-5.  The adjoint with the zones on satisfies the transpose identity
against the oracle's tangent-linear step.  Grids of 24 x 20 x 32 span several
14 x 6 x 6 tiles with ragged tails in r and theta.
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle
import synthetic as syn
from tests.parity import jitter, rel_l1

pytestmark = pytest.mark.gpu

ZONES = (1.25 * 0.5, 0.84 * 2.0, 0.01)


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2207_04252_gb300 import build
    build.build()
    from paper_2207_04252_gb300 import rossbi, workloads
    torch.cuda.init()
    return rossbi, workloads


def _reference(w, steps):
    o = oracle.Oracle(w)
    E0 = oracle.initial_state(o)
    o.set_damping(*ZONES)
    E, _, dts = o.run(E0.copy(), steps=steps)
    assert o.take_status() == 0
    o.set_damping(*ZONES[:2], 0.0)
    E_off, _, _ = o.run(E0.copy(), dts=dts)
    return o, E, E_off, dts


@pytest.fixture(scope="module", params=["disc", "vortex"])
def reference(request):
    if request.param == "disc":
        w = syn.scaled(syn.DISC_NOISE, 24, 20, 32)
        return (w,) + _reference(w, 40)
    w = syn.scaled(syn.VORTEX, 24, 20, 32)
    return (w,) + _reference(w, 20)  # the oracle's own drift: 3.4e-13 after 20 steps, 1e-11 after 25


@pytest.mark.parametrize("form", ["fp64", "fp64_pert", "fp32_pert"])
def test_damping_parity(lib, reference, form):
    R, W = lib
    w, o, E_ref, E_off, dts = reference
    prec = {"fp64": R.ROSSBI_FP64, "fp64_pert": R.ROSSBI_FP64_PERT, "fp32_pert": R.ROSSBI_FP32_PERT}[form]
    tol = 1e-5 if form == "fp32_pert" else 1e-12
    g = W.Grid(w, precision=prec)
    g.set_damping(ZONES)
    s = g.initial_state("cuda")
    for dt in dts:
        g.step(s, dt=dt)
    assert g.take_status() == 0
    V = o.volumes()
    errs = rel_l1(g.full_state(s), E_ref, V)
    assert all(e <= tol for e in errs.values()), errs
    # with the zones off the run lands far from the damped one
    Eq = o.equilibrium_state()
    dev = np.abs(E_off - E_ref)[4].sum() / np.abs(E_ref - Eq)[4].sum()
    assert dev > 1e3 * tol, dev
    g.close()


def test_equilibrium_stays_bit_exact(lib):
    import torch
    R, W = lib
    w = replace(syn.scaled(syn.DISC_NOISE, 24, 20, 32), noise_amp=0.0)
    g = W.Grid(w)
    g.set_damping(ZONES)
    s = g.initial_state("cuda")
    s0 = s.clone()
    dt = g.cfl_dt(s)
    for _ in range(5):
        g.step(s, dt=dt)
    assert g.take_status() == 0
    assert bool(torch.equal(s, s0))
    g.close()


def test_adjoint_with_damping(lib):
    """<lam, J delta> (oracle tangent-linear step) = <J^T lam, delta> (GPU
    adjoint) with the zones on, on a jittered bi-fluid vortex."""
    import torch
    R, W = lib
    w = syn.scaled(syn.VORTEX, 20, 18, 32)
    o = oracle.Oracle(w)
    o.set_damping(*ZONES)
    rng = np.random.default_rng(4)
    E0 = jitter(oracle.initial_state(o), w.gamma, rng, 1e-3)
    dt = o.cfl_dt(E0)
    scale = np.abs(E0).mean(axis=(1, 2, 3), keepdims=True) + 1e-30
    lam = rng.standard_normal(E0.shape) / scale
    delta = rng.standard_normal(E0.shape) * scale
    _, t = o.step_tlm(E0, delta, dt)
    assert o.take_status() == 0
    g = W.Grid(w)
    g.set_damping(ZONES)
    lam_d = torch.from_numpy(lam).cuda().contiguous()
    g.adjoint_step(torch.from_numpy(E0).cuda().contiguous(), dt, lam_d)
    assert g.take_status() == 0
    lhs, rhs = float((lam * t).sum()), float((lam_d.cpu().numpy() * delta).sum())
    assert abs(lhs - rhs) <= 1e-12 * float(np.abs(lam * t).sum()), (lhs, rhs)
    # and the zones matter to the adjoint: without them the cotangent differs
    g.set_damping(None)
    lam_off = torch.from_numpy(lam).cuda().contiguous()
    g.adjoint_step(torch.from_numpy(E0).cuda().contiguous(), dt, lam_off)
    r = np.abs(lam_off.cpu().numpy() - lam_d.cpu().numpy()).sum() / np.abs(lam_d.cpu().numpy()).sum()
    assert r > 1e-6, r
    g.close()


def test_argument_errors(lib):
    R, W = lib
    g = W.Grid(syn.scaled(syn.DISC_NOISE, 24, 20, 32))
    for bad in ((0.4, 1.6, 1.0), (0.6, 2.5, 1.0), (1.5, 1.0, 1.0), (0.6, 1.6, 0.0), (0.6, 1.6, float("nan"))):
        with pytest.raises(R.RossbiError) as e:
            g.set_damping(bad)
        assert e.value.code == R.ROSSBI_ERR_ARG
    g.set_damping(None)
    g.close()
    box = W.Grid(syn.scaled(syn.SOD, 16, 2, 2))
    with pytest.raises(R.RossbiError):
        box.set_damping((0.2, 0.8, 1.0))
    box.set_damping(None)
    box.close()


# ---------------------------------------------------------------- vertical sheared damped boundary (reading R21)
ZONE_Z = (0.06, 0.01)


def _reference_z(w, steps, with_radial):
    o = oracle.Oracle(w)
    E0 = oracle.initial_state(o)
    if with_radial:
        o.set_damping(*ZONES)
    o.set_vertical_damping(*ZONE_Z)
    E, _, dts = o.run(E0.copy(), steps=steps)
    assert o.take_status() == 0
    o.set_vertical_damping(ZONE_Z[0], 0.0)
    E_off, _, _ = o.run(E0.copy(), dts=dts)
    return o, E, E_off, dts


@pytest.fixture(scope="module", params=["disc", "vortex_with_radial"])
def reference_z(request):
    if request.param == "disc":
        w = syn.scaled(syn.DISC_NOISE, 24, 20, 32)
        return (w, False) + _reference_z(w, 40, False)
    w = syn.scaled(syn.VORTEX, 24, 20, 32)
    return (w, True) + _reference_z(w, 15, True)


@pytest.mark.parametrize("form", ["fp64", "fp64_pert", "fp32_pert"])
def test_vertical_damping_parity(lib, reference_z, form):
    R, W = lib
    w, with_radial, o, E_ref, E_off, dts = reference_z
    prec = {"fp64": R.ROSSBI_FP64, "fp64_pert": R.ROSSBI_FP64_PERT, "fp32_pert": R.ROSSBI_FP32_PERT}[form]
    tol = 1e-5 if form == "fp32_pert" else 1e-12
    g = W.Grid(w, precision=prec)
    if with_radial:
        g.set_damping(ZONES)
    g.set_vertical_damping(ZONE_Z)
    s = g.initial_state("cuda")
    for dt in dts:
        g.step(s, dt=dt)
    assert g.take_status() == 0
    V = o.volumes()
    errs = rel_l1(g.full_state(s), E_ref, V)
    assert all(e <= tol for e in errs.values()), errs
    Eq = o.equilibrium_state()
    dev = np.abs(E_off - E_ref)[4].sum() / np.abs(E_ref - Eq)[4].sum()
    assert dev > 20 * tol, dev
    g.close()


def test_vertical_damping_adjoint_and_equilibrium(lib):
    import torch
    R, W = lib
    w = syn.scaled(syn.VORTEX, 20, 18, 32)
    o = oracle.Oracle(w)
    o.set_damping(*ZONES)
    o.set_vertical_damping(*ZONE_Z)
    rng = np.random.default_rng(5)
    E0 = jitter(oracle.initial_state(o), w.gamma, rng, 1e-3)
    dt = o.cfl_dt(E0)
    scale = np.abs(E0).mean(axis=(1, 2, 3), keepdims=True) + 1e-30
    lam = rng.standard_normal(E0.shape) / scale
    delta = rng.standard_normal(E0.shape) * scale
    _, t = o.step_tlm(E0, delta, dt)
    assert o.take_status() == 0
    g = W.Grid(w)
    g.set_damping(ZONES)
    g.set_vertical_damping(ZONE_Z)
    lam_d = torch.from_numpy(lam).cuda().contiguous()
    g.adjoint_step(torch.from_numpy(E0).cuda().contiguous(), dt, lam_d)
    assert g.take_status() == 0
    lhs, rhs = float((lam * t).sum()), float((lam_d.cpu().numpy() * delta).sum())
    assert abs(lhs - rhs) <= 1e-12 * float(np.abs(lam * t).sum()), (lhs, rhs)
    # an undisturbed disc stays bit for bit
    g2 = W.Grid(replace(syn.scaled(syn.DISC_NOISE, 24, 20, 32), noise_amp=0.0))
    g2.set_vertical_damping(ZONE_Z)
    s = g2.initial_state("cuda")
    s0 = s.clone()
    dt2 = g2.cfl_dt(s)
    for _ in range(5):
        g2.step(s, dt=dt2)
    assert bool(torch.equal(s, s0))
    for bad in ((-0.01, 1.0), (0.2, 1.0), (0.06, 0.0), (0.06, float("inf"))):
        with pytest.raises(R.RossbiError) as e:
            g2.set_vertical_damping(bad)
        assert e.value.code == R.ROSSBI_ERR_ARG
    g2.set_vertical_damping(None)
    g.close()
    g2.close()
