"""Gradients through many steps: the checkpointed discrete adjoint behind torch.autograd.

``run_steps(grid, E0, dts, stokes)`` advances an FP64 state through
len(dts) steps of the given lengths (a frozen CFL sequence) and is
differentiable in the initial state and the Stokes number.  The forward pass
keeps a copy of the state every ``every`` steps (revolve-style checkpoints);
the backward pass walks the segments from the last one, recomputes each
segment's states from its checkpoint and runs ``rossbi_adjoint_step`` back
through them.  Memory: ceil(K / every) + every states; extra work: one
forward run.

``vortex_core_weights`` builds dJ/dE for the objective "dust mass inside the
vortex core", J = sum over cells with ((r - r_v) / s_r)^2 + (r_v dtheta / s_t)^2
<= 1 (all z) of V rho_d, so that J = (weights * E).sum().
"""
import functools
import math

import numpy as np
import torch

import synthetic as syn

from . import rossbi as R


@functools.lru_cache(maxsize=None)
def _revolve_cost(n, s):
    """(forward steps, first split) to reverse n steps from a stored start
    state with s more snapshots: the best split m advances m steps, stores a
    snapshot, reverses the last n - m steps with s - 1 snapshots and the first
    m with s (binomial checkpointing; with no snapshot left every step is
    recomputed from the start)."""
    if n <= 1:
        return 0, 0
    if s == 0:
        return n * (n - 1) // 2, 0
    best = None
    for m in range(1, n):
        c = m + _revolve_cost(n - m, s - 1)[0] + _revolve_cost(m, s)[0]
        if best is None or c < best[0]:
            best = (c, m)
    return best


class _Steps(torch.autograd.Function):
    @staticmethod
    def forward(ctx, E0, stokes, grid, dts, every, agrid, snapshots):
        law = grid.dust[1] if grid.dust else 0
        grid.dust = (float(stokes), law) if grid.dust else None
        agrid.dust = grid.dust
        E = E0.detach().clone().contiguous()
        ckpts = []
        for n, dt in enumerate(dts):
            if snapshots is None and n % every == 0:
                ckpts.append(E.clone())
            elif snapshots is not None and n == 0:
                ckpts.append(E.clone())
            grid.step(E, dt=dt)
        ctx.grid, ctx.agrid, ctx.dts, ctx.every, ctx.ckpts = grid, agrid, list(dts), every, ckpts
        ctx.snapshots = snapshots
        ctx.in_dtype = E0.dtype
        ctx.forward_steps = 0
        return E

    @staticmethod
    def backward(ctx, lam_out):
        grid, agrid, dts, every = ctx.grid, ctx.agrid, ctx.dts, ctx.every
        lam = lam_out.detach().to(torch.float64).clone().contiguous()
        R.rossbi_adjoint_dstokes(agrid.h, reset=True)
        K = len(dts)
        full = _full_state_fn(grid)

        def advance(E, n0, n1):
            E = E.clone()
            for n in range(n0, n1):
                grid.step(E, dt=dts[n])
            ctx.forward_steps += n1 - n0
            return E

        def reverse(E_start, n0, n1, snaps):
            """Adjoint steps n1-1 .. n0, given the state at step n0."""
            if n1 - n0 == 1:
                agrid.adjoint_step(full(E_start), dts[n0], lam)
                return
            if snaps == 0:
                for n in reversed(range(n0, n1)):
                    agrid.adjoint_step(full(advance(E_start, n0, n)), dts[n], lam)
                return
            m = n0 + _revolve_cost(n1 - n0, snaps)[1]
            reverse(advance(E_start, n0, m), m, n1, snaps - 1)
            reverse(E_start, n0, m, snaps)

        if ctx.snapshots is not None:
            reverse(ctx.ckpts[0], 0, K, ctx.snapshots)
        else:
            for s in reversed(range(len(ctx.ckpts))):
                start, end = s * every, min((s + 1) * every, K)
                states = [ctx.ckpts[s]]
                for n in range(start, end - 1):
                    states.append(advance(states[-1], n, n + 1))
                for n in reversed(range(start, end)):
                    agrid.adjoint_step(full(states[n - start]), dts[n], lam)
        dst = R.rossbi_adjoint_dstokes(agrid.h, reset=True) if grid.dust else 0.0
        ctx.ckpts = None
        _last_backward["forward_steps"] = ctx.forward_steps
        return lam.to(ctx.in_dtype), torch.tensor(dst, dtype=torch.float64), None, None, None, None, None


# Steps recomputed by the most recent backward sweep (for tests and measurement).
_last_backward = {"forward_steps": 0}


def _full_state_fn(grid):
    """State of `grid` -> the FP64 full state the adjoint linearises about."""
    if grid.precision == R.ROSSBI_FP64:
        return lambda s: s
    E0 = torch.zeros(grid.shape, dtype=torch.float64, device="cuda")
    if grid.w.disc is not None:
        E0[:5] = torch.from_numpy(grid.equilibrium()).cuda()[:, :, None, :]

    def full(s):
        return (E0 + s.to(torch.float64)).contiguous()
    return full


def run_steps(grid, E0, dts, stokes=None, every=20, adjoint_grid=None, snapshots=None):
    """E^K from E^0 (a state of `grid`, (nf, nz, nth, nr) on the device)
    through the steps dts; differentiable in E0 and in `stokes` (a 0-d float64
    tensor; default: the workload's Stokes number, not tracked).

    Checkpoints: by default the state every `every` steps (segments are
    recomputed once in the backward sweep).  With `snapshots` = s, binomial
    (revolve) checkpointing instead: the forward run keeps only E^0 and the
    backward sweep holds at most s + 1 states, recomputing the fewest forward
    steps a schedule with s snapshots allows.

    An FP64 grid is its own adjoint grid.  For a perturbation-form grid (the
    state is E' = E - E0) the forward run and the checkpoints stay in that
    form and `adjoint_grid`, an FP64 grid of the same workload, supplies the
    FP64 adjoint steps, linearised about E0 + E' of the recomputed states."""
    if stokes is None:
        stokes = torch.tensor(grid.w.stokes, dtype=torch.float64)
    agrid = grid if grid.precision == R.ROSSBI_FP64 else adjoint_grid
    if agrid is None or agrid.precision != R.ROSSBI_FP64:
        raise R.RossbiError(R.ROSSBI_ERR_ARG, "run_steps: a perturbation-form grid needs an FP64 adjoint_grid")
    if snapshots is not None and int(snapshots) < 0:
        raise R.RossbiError(R.ROSSBI_ERR_ARG, "run_steps: snapshots must be >= 0")
    return _Steps.apply(E0, stokes, grid, list(dts), int(every), agrid,
                        None if snapshots is None else int(snapshots))


def revolve_forward_steps(n, snapshots):
    """Forward steps the revolve schedule recomputes to reverse n steps."""
    return _revolve_cost(int(n), int(snapshots))[0]


def cfl_sequence(grid, E0, steps):
    """The CFL step lengths of a plain forward run of `steps` steps from E0."""
    E = E0.clone()
    dt = grid.cfl_dt(E)
    dts = []
    for _ in range(steps):
        dts.append(dt)
        dt = grid.step(E, dt=dt, want_next_dt=True)
    return dts


def vortex_core_weights(grid, vortex=0):
    """dJ/dE of J = dust mass inside the core ellipse of a vortex (all z)."""
    w = grid.w
    rv, thv = w.vortices[vortex]
    sigma0, beta_sigma, T0, beta_T = w.disc
    omk = math.sqrt(w.gm / rv ** 3)
    s_r = w.vortex_width_h * math.sqrt(2.0 * T0 * rv ** beta_T) / omk
    s_t = w.vortex_chi * s_r
    r = grid.centres(0)[None, :]
    th = grid.centres(1)[:, None]
    dth = np.mod(th - thv + math.pi, 2.0 * math.pi) - math.pi
    inside = ((r - rv) / s_r) ** 2 + (rv * dth / s_t) ** 2 <= 1.0
    f = w.x0[0] * (w.x1[0] / w.x0[0]) ** (np.arange(w.nr + 1) / w.nr)
    dth_c = (w.x1[1] - w.x0[1]) / w.nth
    dz = (w.x1[2] - w.x0[2]) / w.nz
    V = 0.5 * (f[1:] ** 2 - f[:-1] ** 2) * dth_c * dz
    W = np.zeros(grid.shape)
    W[syn.F_DRHO] = (inside * V[None, :])[None, :, :]
    return torch.from_numpy(W)
