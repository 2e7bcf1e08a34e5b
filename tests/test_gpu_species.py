"""Several dust species on the GPU (Sect. 5.4's multi-fluid approach, the
drag law of Sect. 2.9 per species; reading R20) against the oracle.

The bi-fluid vortex with three species of Stokes numbers St x (1, 0.3, 3),
each an equal share of the dust, runs on the oracle's dt sequence: FP64 and
the FP64 perturbation form <= 1e-12, FP32 <= 1e-5 (relative L1 per conserved
quantity, the dust groups summed over species), beside the element-wise
measure.  Four species put the FP64-state kernels on their thin (two z
cells) tiles.  Two half-density twins of one species reproduce the single
fluid.  The paper's conservative reconstruction is compared over 15 steps
(the oracle's own drift on this vortex is ~1e-13 there; see
test_gpu_parity.py).
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle
import synthetic as syn
from tests.parity import elementwise, rel_l1

pytestmark = pytest.mark.gpu

STEPS = 15


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2207_04252_gb300 import build
    build.build()
    from paper_2207_04252_gb300 import rossbi, workloads
    torch.cuda.init()
    return rossbi, workloads


def _groups(E):
    """Gas fields and the species' dust fields summed into one dust fluid
    (nf = 9), so that rel_l1's groups cover every species."""
    nd = (E.shape[0] - 5) // 4
    out = np.zeros((9,) + E.shape[1:])
    out[:5] = E[:5]
    for s in range(nd):
        out[5:9] += np.abs(E[5 + 4 * s:9 + 4 * s])
    return out


def _l1(E_test, E_ref, V):
    """Relative L1 per conserved quantity; each dust species is its own fluid,
    so the dust groups sum the species' errors and magnitudes."""
    nd = (E_ref.shape[0] - 5) // 4
    out = rel_l1(E_test[:5], E_ref[:5], V)
    Vb = V[None, None, :]
    for name, offs in (("dust_mass", (3,)), ("dust_momentum", (0, 1, 2))):
        num = sum((Vb * np.abs(E_test[5 + 4 * s + c] - E_ref[5 + 4 * s + c])).sum() for s in range(nd) for c in offs)
        den = sum((Vb * np.abs(E_ref[5 + 4 * s + c])).sum() for s in range(nd) for c in offs)
        out[name] = float(num / den)
    return out


def _workload(nd, factors, n=(20, 18, 32)):
    return replace(syn.scaled(syn.VORTEX, *n), n_dust=nd, dust_stokes_factors=factors)


CASES = [("three", 3, (1.0, 0.3, 3.0), (20, 18, 32)), ("four_thin_tiles", 4, (1.0, 0.5, 2.0, 8.0), (17, 13, 33)),
         ("two", 2, (1.0, 0.1), (29, 13, 32))]


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def reference(request):
    name, nd, factors, n = request.param
    w = _workload(nd, factors, n)
    o = oracle.Oracle(w)
    E0 = oracle.initial_state(o)
    E, _, dts = o.run(E0.copy(), steps=STEPS)
    assert o.take_status() == 0
    return w, o, E0, E, dts


@pytest.mark.parametrize("form", ["fp64", "fp64_pert", "fp32_pert"])
def test_species_parity(lib, reference, form):
    import torch
    R, W = lib
    w, o, E0, E_ref, dts = reference
    prec = {"fp64": R.ROSSBI_FP64, "fp64_pert": R.ROSSBI_FP64_PERT, "fp32_pert": R.ROSSBI_FP32_PERT}[form]
    tol, el_tol = (1e-5, 1e-2) if form == "fp32_pert" else (1e-12, 1e-8)
    g = W.Grid(w, precision=prec)
    assert g.nf == 5 + 4 * w.n_dust
    s = g.initial_state()
    # the two sides build the initial state each from its own equilibrium and
    # recipe: equal to rounding (float storage in the FP32 form)
    scale = np.abs(E0).max(axis=(1, 2, 3), keepdims=True)
    err0 = np.abs(g.full_state(s) - E0) / np.where(scale > 0, scale, 1.0)
    assert err0.max() <= (1e-6 if form == "fp32_pert" else 1e-12), err0.max()
    for dt in dts:
        g.step(s, dt=dt)
    assert g.take_status() == 0
    E = g.full_state(s)
    errs = _l1(E, E_ref, o.volumes())
    el = elementwise(E, E_ref, g.equilibrium())
    print(form, w.n_dust, "species", {k: f"{v:.1e}" for k, v in errs.items()},
          {k: (f"{r:.1e}", at) for k, (r, at) in el.items()})
    assert all(e <= tol for e in errs.values()), errs
    assert all(r <= el_tol for r, _ in el.values()), el
    # the species really differ: with every factor 1 the dust lands elsewhere
    if form == "fp64":
        w1 = replace(w, dust_stokes_factors=(1.0,) * w.n_dust)
        g1 = W.Grid(w1, precision=prec)
        s1 = g1.initial_state()
        for dt in dts:
            g1.step(s1, dt=dt)
        off = _l1(g1.full_state(s1), E_ref, o.volumes())
        assert off["dust_momentum"] > 1e3 * tol, off
        g1.close()
    g.close()
    del s
    torch.cuda.empty_cache()


def test_half_density_twins_equal_one_fluid(lib):
    """Two identical species of half the density each: the gas evolves as with
    the single fluid, and each twin carries half of its dust (1e-12, FP64;
    the two drag closed forms differ only in rounding)."""
    import torch
    R, W = lib
    w1 = syn.scaled(syn.VORTEX, 20, 18, 32)
    w2 = replace(w1, n_dust=2, dust_stokes_factors=(1.0, 1.0))
    g1, g2 = W.Grid(w1), W.Grid(w2)
    s1 = g1.initial_state()
    E = s1.cpu().numpy()
    E2 = np.zeros((13,) + E.shape[1:])
    E2[:5] = E[:5]
    E2[5:9] = 0.5 * E[5:9]
    E2[9:13] = 0.5 * E[5:9]
    s2 = torch.from_numpy(E2).cuda()
    dt = g1.cfl_dt(s1)
    assert g2.cfl_dt(s2) == pytest.approx(dt, rel=1e-15)
    for _ in range(STEPS):
        g2.step(s2, dt=dt)
        dt = g1.step(s1, dt=dt, want_next_dt=True)
    a, b = s1.cpu().numpy(), s2.cpu().numpy()
    V = np.ones(w1.nr)
    assert max(rel_l1(b[:5], a[:5], V).values()) <= 1e-12
    for half in (b[5:9], b[9:13]):
        assert np.abs(2.0 * half - a[5:9]).max() <= 1e-12 * np.abs(a[5:9]).max()
    g1.close()
    g2.close()


def test_species_cfl_and_sums(lib):
    R, W = lib
    w = _workload(3, (1.0, 0.3, 3.0), (40, 30, 32))
    o = oracle.Oracle(w)
    E = oracle.initial_state(o)
    for prec, rtol_dt, rtol_s in ((R.ROSSBI_FP64, 1e-14, 1e-13), (R.ROSSBI_FP64_PERT, 1e-13, 1e-13),
                                  (R.ROSSBI_FP32_PERT, 2e-6, 1e-7)):
        g = W.Grid(w, precision=prec)
        s = g.initial_state()
        assert g.cfl_dt(s) == pytest.approx(o.cfl_dt(E), rel=rtol_dt)
        ref = o.sums(E)
        np.testing.assert_allclose(g.sums(s), ref, rtol=rtol_s, atol=rtol_s * np.abs(ref).max())
        g.close()


def test_species_indirect_moments(lib):
    """Every species' density enters the disc moments of Sect. 2.10."""
    R, W = lib
    w = _workload(3, (1.0, 0.3, 3.0), (24, 20, 32))
    o = oracle.Oracle(w)
    o.set_indirect(1.0)
    import torch
    from tests.test_oracle_indirect import bump
    g = W.Grid(w)
    E = bump(g.full_state(g.initial_state()), g.centres(0), g.centres(1), g.centres(2))  # gas and species 0
    th = g.centres(1)[None, :, None]
    for b, c in ((9, 4.0), (13, 5.5)):  # the other species off centre elsewhere
        E[b:b + 4] *= (1.0 + 0.3 * np.exp(-(np.angle(np.exp(1j * (th - c))) / 0.5) ** 2))[None]
    s = torch.from_numpy(E).cuda()
    ab = g.indirect_moments(s)
    ref = o.indirect(E)
    assert np.abs(ab - ref).max() <= 1e-12 * np.hypot(*ref), (ab, ref)
    # every species counts: without the third species' excess the moments move
    E2 = E.copy()
    E2[13:17] = bump(g.full_state(g.initial_state()), g.centres(0), g.centres(1), g.centres(2))[13:17]
    assert np.abs(o.indirect(E2) - ref).max() > 1e-3 * np.hypot(*ref)
    g.close()


def test_species_argument_errors(lib):
    import torch
    R, W = lib
    w = _workload(3, (1.0, 0.3, 3.0), (16, 12, 16))
    g = W.Grid(w)
    for bad in ((1.0, 0.3), (2.0, 0.3, 3.0), (1.0, 0.0, 3.0), (1.0, float("nan"), 3.0), (1.0, 1.0, 1.0, 1.0)):
        with pytest.raises(R.RossbiError) as e:
            R.rossbi_set_dust_species(g.h, bad)
        assert e.value.code == R.ROSSBI_ERR_ARG
    s = g.initial_state()
    lam = torch.zeros_like(s)
    with pytest.raises(R.RossbiError) as e:  # the adjoint carries one species
        g.adjoint_step(s, 1e-4, lam)
    assert e.value.code == R.ROSSBI_ERR_UNSUPPORTED
    g.close()
    gas = W.Grid(syn.scaled(syn.DISC_NOISE, 16, 12, 16))
    with pytest.raises(R.RossbiError):
        R.rossbi_set_dust_species(gas.h, (1.0,))
    gas.close()
