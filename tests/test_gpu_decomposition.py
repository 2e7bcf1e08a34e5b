"""The decomposition of Sect. 3.1 on one GPU: a grid split in theta into two
sub-domain grids, each holding its owned rows plus four halo rows on each
side, stepped separately and joined by a halo exchange after every step
(rossbi_pack_theta_rows into a contiguous device buffer, then
rossbi_unpack_theta_rows, the two kernels a multi-GPU run would put around
its send and receive).  The step length is the minimum of the sub-domains'
CFL minima, taken after the exchange.  The owned rows must equal the
undivided grid's bit for bit: the exchange changes no arithmetic (four rows
are what two RK stages of a 2-cell stencil need; tests/test_decomposition.py
shows on the oracle that three are not enough).

The sub-domains have 24 owned + 8 halo = 32 rows, so that their dtheta,
computed by the library as (theta extent) / 32, is the whole grid's 2 pi / 48
bit for bit (a factor of 32 is exact).
"""
from dataclasses import replace
import math

import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu

NTH, OWN, H = 48, 24, 4


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2207_04252_gb300 import build
    build.build()
    from paper_2207_04252_gb300 import rossbi, workloads
    torch.cuda.init()
    return rossbi, workloads


def _sub(w):
    dth = (w.x1[1] - w.x0[1]) / w.nth
    n = OWN + 2 * H
    return replace(w, name=w.name + "@sub", nth=n, x0=(w.x0[0], 0.0, w.x0[2]), x1=(w.x1[0], n * dth, w.x1[2]))


def _rows(s):
    """Global theta rows held by sub-domain s (its row 0 first)."""
    return [(s * OWN - H + j) % NTH for j in range(OWN + 2 * H)]


@pytest.mark.parametrize("wl", ["vortex", "disc"])
@pytest.mark.parametrize("form", ["fp64", "fp32_pert"])
def test_two_subdomains_bit_exact(lib, form, wl):
    import torch
    R, W = lib
    base = syn.VORTEX if wl == "vortex" else syn.DISC_NOISE
    w = syn.scaled(base, 20, NTH, 32)
    prec = R.ROSSBI_FP64 if form == "fp64" else R.ROSSBI_FP32_PERT
    gf = W.Grid(w, precision=prec)
    ws = _sub(w)
    assert (ws.x1[1] - ws.x0[1]) / ws.nth == (w.x1[1] - w.x0[1]) / w.nth
    subs = [W.Grid(ws, precision=prec) for _ in range(2)]
    F = gf.initial_state()
    S = [F[:, :, _rows(s), :].contiguous() for s in range(2)]
    nf, nz, nr = gf.nf, w.nz, w.nr
    buf = torch.empty(nf * nz * H * nr, dtype=gf.dtype, device="cuda")

    def exchange():
        # (source sub, its first row, destination sub, its first row), four rows each
        for src, js, dst, jd in ((1, OWN, 0, 0), (1, H, 0, OWN + H), (0, OWN, 1, 0), (0, H, 1, OWN + H)):
            R.rossbi_pack_theta_rows(subs[src].h, S[src], js, H, buf)
            R.rossbi_unpack_theta_rows(subs[dst].h, S[dst], jd, H, buf)

    for n in range(10):
        dt = gf.cfl_dt(F)
        dt_sub = min(g.cfl_dt(s) for g, s in zip(subs, S))
        assert dt_sub == dt, (n, dt_sub, dt)
        gf.step(F, dt=dt)
        for g, s in zip(subs, S):
            g.step(s, dt=dt)
        exchange()
    for g in [gf] + subs:
        assert g.take_status() == R.ROSSBI_OK
    full = F.cpu().numpy()
    for s in range(2):
        own = S[s][:, :, H:H + OWN, :].cpu().numpy()
        assert np.array_equal(own, full[:, :, s * OWN:(s + 1) * OWN, :]), s
        halo = S[s].cpu().numpy()[:, :, list(range(H)) + list(range(H + OWN, OWN + 2 * H)), :]
        rows = [_rows(s)[j] for j in list(range(H)) + list(range(H + OWN, OWN + 2 * H))]
        assert np.array_equal(halo, full[:, :, rows, :]), s  # the exchanged halos too
    for g in [gf] + subs:
        g.close()


def test_theta_rows_round_trip_and_errors(lib):
    import torch
    R, W = lib
    w = syn.scaled(syn.VORTEX, 20, 18, 16)
    g = W.Grid(w)
    s = g.initial_state()
    buf = torch.empty(g.nf * w.nz * 5 * w.nr, dtype=torch.float64, device="cuda")
    R.rossbi_pack_theta_rows(g.h, s, 7, 5, buf)
    ref = s[:, :, 7:12, :].contiguous().reshape(-1)
    assert torch.equal(buf, ref)
    t = torch.zeros_like(s)
    R.rossbi_unpack_theta_rows(g.h, t, 7, 5, buf)
    assert torch.equal(t[:, :, 7:12, :], s[:, :, 7:12, :]) and int(torch.count_nonzero(t[:, :, :7])) == 0
    for j0, rows in ((-1, 2), (17, 2), (0, 0), (0, 19)):
        with pytest.raises(R.RossbiError) as e:
            R.rossbi_pack_theta_rows(g.h, s, j0, rows, buf)
        assert e.value.code == R.ROSSBI_ERR_ARG
    g.close()
