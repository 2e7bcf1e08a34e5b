"""The oracle's non-axisymmetric dynamics pinned by the Rossby wave
instability (Sect. 4.3): the mode m = 4 of the bumped disc grows in the
oracle at a rate consistent with the eigenvalues of the linearised equations
(tests/rwi_linear.py), a computation that shares nothing with the scheme.

The case is kept small for the CPU: 2-D (one midplane z cell), the annulus
r in [0.75, 1.35] in its equal-Mach frame with wave-killing zones at 0.8 and
1.28, and a quarter of the circle (theta periodic over pi/2, which holds
mode 4 as its fundamental), 64 x 24 cells.  At this resolution (2.7 cells per
bump width) the scheme's dissipation costs the mode about 30 % of its rate;
the GPU runs of the same scheme converge to the linear rate with the mesh
(0.83, 0.97, 0.99 of it at 128, 256, 512 cells a side).  A sign or metric
mistake in the azimuthal or radial terms stops the growth or moves the rate
far outside the band.  The run takes the primitive-departure option, which
grows at 0.715 of the linear rate here (option 2, the pressure departure in
place of the energy one, at 0.716 on the same case); the conservative
reading of the paper turns this coarse run non-physical (its high-Mach
instability) and is held to the rate on the GPU instead, on the same
annulus at 154 x 256 cells.
"""
from dataclasses import replace
import math

import numpy as np

import oracle
import synthetic as syn
from tests.rwi_linear import rwi_growth_rate

H = 0.05
R_IN, R_OUT = 0.75, 1.35


def test_rwi_mode_grows_at_the_linear_rate():
    w = replace(syn.RWI, nr=64, nth=24, nz=1, recon=syn.RECON_PRIMITIVE,
                x0=(R_IN, 0.0, -0.5 * H), x1=(R_OUT, 0.5 * math.pi, 0.5 * H),
                bc_lo=(syn.BC_EQUILIBRIUM, syn.BC_PERIODIC, syn.BC_PERIODIC),
                bc_hi=(syn.BC_EQUILIBRIUM, syn.BC_PERIODIC, syn.BC_PERIODIC),
                omega_frame=syn.workloads.equal_mach_frame(R_IN, R_OUT))
    o = oracle.Oracle(w)
    o.set_damping(0.8, 1.28, 1.0)
    E = oracle.initial_state(o)
    r, _ = o.coords(0)
    th, _ = o.coords(1)
    sel = np.abs(r - w.rwi_r0) < 0.03
    ph = np.exp(-1j * w.rwi_mode * th)

    def amp(E):
        vr = E[syn.F_MU, 0] / E[syn.F_RHO, 0]
        c = (vr * ph[:, None]).sum(axis=0) * 2.0 / w.nth
        return float(np.sqrt(np.mean(np.abs(c[sel]) ** 2)))

    t_end, t, nt = 50.0, 0.0, 0.5
    hist = [(0.0, amp(E))]
    for _ in range(12000):             # the run takes ~7 500 steps; a collapsing step fails
        if t >= t_end:
            break
        dt = o.cfl_dt(E)
        E = o.step(E, dt)
        t += dt
        if t >= nt:
            hist.append((t, amp(E)))
            nt += 0.5
    assert o.take_status() == 0
    assert t >= t_end, t
    h = np.array(hist)
    late = h[:, 0] >= 0.5 * t_end
    rate = float(np.polyfit(h[late, 0], np.log(h[late, 1]), 1)[0])
    lin = rwi_growth_rate(lambda x: o.eq_prim(x, 0.0), w.rwi_mode, w.rwi_r0, R_IN, R_OUT, n=200)
    print(f"oracle m = 4: fitted {rate:.4f}, linear {lin:.4f}, ratio {rate / lin:.3f}")
    assert lin > 0.1
    assert 0.6 <= rate / lin <= 1.05, (rate, lin)
    assert h[-1, 1] >= 5.0 * h[:, 1].min()
