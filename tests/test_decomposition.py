"""The spatial decomposition of Sect. 3.1, checked on CPU ranks with the oracle.

The library runs one grid per GPU and several GPUs as independent replicas;
this test shows that the step shards the way the paper decomposes it, and
what the exchange step must carry.  Two gloo ranks each own half of the
azimuthal cells (theta is periodic, the paper's first split).  A rank holds
its cells plus a halo of h cells on each side; every other cell holds a
different but physical state (the disc turned by a quarter in theta), so a
result that depends on anything outside the halo comes out different (NaN
would not do: the limiter's comparisons silently drop a NaN slope).  The
global step length is an all-reduce minimum of the ranks' own CFL minima.
Each rank advances its own cells by one RK2 step (the oracle's sampled step,
which evaluates the intermediate state lazily on the stencil it needs), and
the gathered result must equal the undivided step bit for bit.  One stage
reaches two cells each way (parabola of the neighbour, face between them), so
a step needs h = 4; with h = 3 the foreign cells reach the owned ones.
"""
import os
import socket

import numpy as np


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, halo, out):
    import torch
    import torch.distributed as dist

    import oracle
    import synthetic as syn
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = syn.scaled(syn.VORTEX, 12, 16, 16)
        o = oracle.Oracle(w)
        E = oracle.initial_state(o)
        per = w.nth // world
        own = np.arange(rank * per, (rank + 1) * per)
        held = np.unique(np.arange(own[0] - halo, own[-1] + halo + 1) % w.nth)
        # the rank's CFL minimum over its own cells (other columns copy one of them)
        Edt = E.copy()
        Edt[:, :, np.setdiff1d(np.arange(w.nth), own), :] = E[:, :, own[:1], :]
        t = torch.tensor([o.cfl_dt(Edt)], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MIN)
        dt = float(t[0])
        # the rank's view: its cells and halo; everything else foreign
        Eloc = np.roll(E, w.nth // 4, axis=2)
        Eloc[:, :, held, :] = E[:, :, held, :]
        k, j, i = np.meshgrid(np.arange(w.nz), own, np.arange(w.nr), indexing="ij")
        cells = ((k * w.nth + j) * w.nr + i).ravel()
        res = o.step_sampled(Eloc, dt, cells)
        gathered = [None] * world
        dist.all_gather_object(gathered, (cells, res, dt))
        if rank == 0:
            out["parts"] = gathered
            out["undivided_dt"] = o.cfl_dt(E)
            out["undivided"] = o.step(E, o.cfl_dt(E))
            out["shape"] = E.shape
    finally:
        dist.destroy_process_group()


def _run(halo):
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(2, port, halo, out), nprocs=2, join=True)
        return dict(out)


def _assemble(res):
    nf = res["shape"][0]
    flat = np.full((nf, int(np.prod(res["shape"][1:]))), np.nan)
    for cells, vals, _ in res["parts"]:
        flat[:, cells] = vals.T
    return flat.reshape(res["shape"])


def test_two_ranks_with_a_four_cell_halo_reproduce_the_step():
    res = _run(4)
    assert all(p[2] == res["undivided_dt"] for p in res["parts"])  # all-reduce min = global CFL
    E = _assemble(res)
    assert np.array_equal(E, res["undivided"])


def test_a_three_cell_halo_is_not_enough():
    res = _run(3)
    assert not np.array_equal(_assemble(res), res["undivided"])
