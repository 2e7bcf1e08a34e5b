"""The Rossby-wave-instability workload (Sect. 4.3) on the GPU.

The equilibrium carries the density bump (rho and P x (1 + delta G), G a
Gaussian at r0 = 1, v_theta0 in radial balance with it); the run evolves the
seed v_r = eps v_theta0 sin(m theta) G.

Parity: the RWI disc against the oracle over 100 steps at 32x48x32, all three
forms (FP64 and the FP64 perturbation form <= 1e-12, FP32 <= 1e-5; the oracle
drifts from a 1e-15 input perturbation by 4e-14 over these 100 steps).

Long runs (reported, not pinned): the mode-m amplitude of v_r on the midplane
ring at r0 every 500 steps, in the FP32 form on the 128x256x16 workload.  The
primitive-departure option stays physical over 30 000 steps (t = 80, about
13 orbits at r0) and the paper's conservative reconstruction over 5 000 (in
this frame it turns non-physical after 7 000 to 12 500 steps, t = 19 to 34,
depending on the seeded mode, in 2-D as in 3-D).  Neither run shows
the instability's growth: the seed decays for every bump tried (delta up to
2, Delta_r = H and 2H, grids up to 512 x 512 in 2-D), so growth rates are not
reproduced and the test asserts none.
"""
from dataclasses import replace
import math

import numpy as np
import pytest

import oracle
import synthetic as syn
from tests.parity import elementwise, rel_l1

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
    w = syn.scaled(syn.RWI, 32, 48, 32, steps=100)
    o = oracle.Oracle(w)
    E, _, dts = o.run(oracle.initial_state(o), steps=100)
    assert o.take_status() == 0
    return w, o, E, dts


@pytest.mark.parametrize("form", ["fp64", "fp64_pert", "fp32_pert"])
def test_rwi_parity(lib, reference, form):
    R, W = lib
    w, o, E_ref, dts = reference
    prec = {"fp64": R.ROSSBI_FP64, "fp64_pert": R.ROSSBI_FP64_PERT, "fp32_pert": R.ROSSBI_FP32_PERT}[form]
    tol, el_tol = (1e-5, 1e-2) if form == "fp32_pert" else (1e-12, 1e-8)
    g = W.Grid(w, precision=prec)
    s = g.initial_state()
    for dt in dts:
        g.step(s, dt=dt)
    assert g.take_status() == 0
    E = g.full_state(s)
    errs = rel_l1(E, E_ref, o.volumes())
    el = elementwise(E, E_ref, g.equilibrium())
    print(form, {k: f"{v:.1e}" for k, v in errs.items()}, {k: (f"{r:.1e}", at) for k, (r, at) in el.items()})
    assert all(e <= tol for e in errs.values()), errs
    assert all(r <= el_tol for r, _ in el.values()), el
    g.close()


def _long_run(R, W, w, steps, every=500):
    """Amplitudes of mode m of v_r on the midplane ring nearest r0 every
    `every` steps of the FP32 form, with the wave-killing zones at 1.25 r_in
    and 0.84 r_out, and the time reached."""
    g = W.Grid(w, precision=R.ROSSBI_FP32_PERT)
    g.set_damping((1.25 * w.x0[0], 0.84 * w.x1[0], 1.0))
    s = g.initial_state()
    E0 = g.equilibrium()
    r = g.centres(0)
    i0 = int(np.argmin(np.abs(r - w.rwi_r0)))
    ks = [w.nz // 2 - 1, w.nz // 2]
    th = g.centres(1)
    m = w.rwi_mode

    def amp():
        sl = s[:, ks][:, :, :, i0].double().cpu().numpy()
        vr = sl[0] / (sl[4] + E0[4][ks, i0][:, None])
        return float(np.abs((vr * np.exp(-1j * m * th)[None]).sum(axis=1)).mean() * 2.0 / w.nth)

    t, dt = 0.0, g.cfl_dt(s)
    hist = [(0, 0.0, amp())]
    for n in range(every, steps + 1, every):
        for _ in range(every):
            t += dt
            dt = g.step(s, dt=dt, want_next_dt=True)
        hist.append((n, t, amp()))
    status = g.take_status()
    g.close()
    return hist, status


@pytest.mark.parametrize("recon,steps", [(syn.RECON_PRIMITIVE, 30000), (syn.RECON_CONSERVATIVE, 5000)],
                         ids=["primitive_30000_steps", "conservative_5000_steps"])
def test_rwi_long_run(lib, recon, steps):
    R, W = lib
    w = replace(syn.RWI, recon=recon)
    hist, status = _long_run(R, W, w, steps)
    print("RWI m = 4 amplitude of v_r at r0 (step, t, amplitude):",
          [(n, f"{t:.2f}", f"{a:.2e}") for n, t, a in hist[:: max(1, len(hist) // 20)]])
    assert status == 0
    assert all(np.isfinite(a) for _, _, a in hist)
