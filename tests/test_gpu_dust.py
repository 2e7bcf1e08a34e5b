"""The analytic dust rates on the GPU, both precision forms: dust settling at
the terminal velocity w_d - w_g = t_s f_z and the Nakagawa-Sekiya-Hayashi
radial drift v_r = -2 St eta v_K / (1 + St^2) (see test_oracle_dust)."""
import numpy as np
import pytest

import oracle
from tests.test_oracle_dust import drift_error, drift_workload, settling_error, settling_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2207_04252_gb300 import build
    build.build()
    from paper_2207_04252_gb300 import rossbi, workloads
    torch.cuda.init()
    return rossbi, workloads


def _run(W, w, prec, steps):
    g = W.Grid(w, precision=prec)
    s = g.initial_state()
    dt = g.cfl_dt(s)
    for _ in range(steps):
        dt = g.step(s, dt=dt, want_next_dt=True)
    E = g.full_state(s)
    g.close()
    return E


@pytest.mark.parametrize("precision", ["fp64", "fp32_pert"])
def test_gpu_dust_settling(lib, precision):
    R, W = lib
    prec = R.ROSSBI_FP64 if precision == "fp64" else R.ROSSBI_FP32_PERT
    w = settling_workload()
    o = oracle.Oracle(w)
    E = _run(W, w, prec, 40)
    assert settling_error(w, E, o.coords(2)[0], o.coords(0)[0]) <= 1e-2


@pytest.mark.parametrize("precision", ["fp64", "fp32_pert"])
def test_gpu_dust_radial_drift(lib, precision):
    R, W = lib
    prec = R.ROSSBI_FP64 if precision == "fp64" else R.ROSSBI_FP32_PERT
    w = drift_workload()
    o = oracle.Oracle(w)
    E = _run(W, w, prec, 400)
    rc = o.coords(0)[0]
    vth = np.array([o.eq_prim(r, 0.0)[1] for r in rc])
    assert drift_error(w, E, rc, vth) <= 1e-2
