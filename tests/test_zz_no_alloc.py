"""rossbi_step_noalloc: the step for callers that cannot allocate device memory.

Checks, through the C ABI, that two calls in a row give the same states and
next dt as rossbi_step (same kernels, scratch in the library's fixed device
array instead of a cudaMalloc'd buffer), with and without the optional
terms, that the calls leave the device's free memory unchanged, and that a
grid whose scratch exceeds the fixed array is refused before anything runs.  Kept in a file collected last so that a
run stopping at the first failure has run every other test first.
"""
import numpy as np
import pytest

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


ZONES = (1.25 * 0.5, 0.84 * 2.0, 0.01)


@pytest.mark.parametrize("option", ["plain", "indirect", "damping", "epstein"])
@pytest.mark.parametrize("precision", ["fp64", "fp32_pert", "fp64_pert"])
def test_noalloc_matches_step(lib, precision, option):
    """The optional terms too: the indirect gravity (whose disc moments are
    summed before each stage into the grid's own tables), the wave-killing
    zones and the Epstein drag law."""
    import torch
    from dataclasses import replace
    from tests.test_gpu_indirect import _lopsided_gpu
    R, W = lib
    prec = {"fp64": R.ROSSBI_FP64, "fp32_pert": R.ROSSBI_FP32_PERT, "fp64_pert": R.ROSSBI_FP64_PERT}[precision]
    w = syn.scaled(syn.VORTEX, 40, 30, 32, steps=2)
    if option == "epstein":
        w = replace(w, drag_law=1)
    g = W.Grid(w, precision=prec)
    if option == "indirect":
        g.set_indirect(0.7)
        a = _lopsided_gpu(g)
    else:
        a = g.initial_state()
    if option == "damping":
        g.set_damping(ZONES)
    b = a.clone()
    # one ordinary step on a throwaway copy first: it loads every kernel the step
    # uses (the CUDA runtime loads kernel code lazily, on first launch, which
    # takes device memory) and allocates the ordinary path's own scratch
    warm = a.clone()
    g.step(warm, dt=g.cfl_dt(warm), want_next_dt=True)
    del warm
    dt_a = dt_b = g.cfl_dt(a)
    for call in range(2):
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        dt_b = R.rossbi_step_noalloc(g.h, b, dt=dt_b, dust=g.dust, want_next_dt=True)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, "rossbi_step_noalloc allocated device memory"
        dt_a = g.step(a, dt=dt_a, want_next_dt=True)
        errs = rel_l1(g.full_state(b), g.full_state(a), np.ones(w.nr))
        assert all(e <= 1e-12 for e in errs.values()), (call, errs)
        assert dt_b == pytest.approx(dt_a, rel=1e-12)
    assert g.take_status() == R.ROSSBI_OK
    g.close()


def test_noalloc_rejects_grid_beyond_capacity(lib):
    R, W = lib
    w = syn.scaled(syn.VORTEX, 128, 128, 64, steps=1)  # 9 x 1,048,576 doubles = 72 MiB > 64 MiB
    g = W.Grid(w, precision=R.ROSSBI_FP64)
    s = g.initial_state()
    before = s.clone()
    with pytest.raises(R.RossbiError) as e:
        R.rossbi_step_noalloc(g.h, s, dt=1e-4, dust=g.dust, want_next_dt=True)
    assert e.value.code == R.ROSSBI_ERR_ARG
    assert bool((s == before).all())
    g.close()
