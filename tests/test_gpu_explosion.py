"""The cylindrical explosion test (Sect. 4.1) on the GPU against the oracle.

FP64 form (the only form that runs a cylindrical grid without a disc): the GPU
follows the oracle's dt sequence to t = 0.1 on a 120 x 12 x 1 polar grid
(ragged 14 x 6 x 6 tiles in r and z) and must agree to <= 1e-12; the solution
must stay exactly independent of theta; the perturbation forms refuse the grid.
"""
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


def test_explosion_parity_and_symmetry(lib):
    R, W = lib
    w = syn.scaled(syn.EXPLOSION, 120, 12, 1, t_end=0.1)
    o = oracle.Oracle(w)
    E_ref, t, dts = o.run(oracle.initial_state(o), t_end=w.t_end)
    assert o.take_status() == 0
    g = W.Grid(w)
    s = g.initial_state("cuda")
    # the GPU's own first CFL step is the oracle's
    assert g.cfl_dt(s) == pytest.approx(dts[0], rel=1e-13)
    for dt in dts:
        g.step(s, dt=dt)
    assert g.take_status() == 0
    E = g.full_state(s)
    errs = rel_l1(E[:5], E_ref[:5], o.volumes())
    assert all(e <= 1e-12 for e in errs.values()), errs
    assert np.array_equal(E, np.broadcast_to(E[:, :, :1, :], E.shape))
    # the waves have moved: the state is far from the initial one
    assert np.abs(E[4] - oracle.initial_state(o)[4]).max() > 0.1
    g.close()


def test_perturbation_forms_refuse_a_grid_without_disc(lib):
    R, W = lib
    w = syn.scaled(syn.EXPLOSION, 40, 8, 1)
    for prec in (R.ROSSBI_FP32_PERT, R.ROSSBI_FP64_PERT):
        with pytest.raises(R.RossbiError) as e:
            W.Grid(w, precision=prec)
        assert e.value.code == R.ROSSBI_ERR_UNSUPPORTED
