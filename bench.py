#!/usr/bin/env python
"""Throughput of the RoSSBi3D time step on GB300, in cell-updates/s.

A step is one full midpoint-RK2 update (two fused stage launches plus the
conservation-sum finalisation) of the whole grid of the synthetic workload,
with the state resident in HBM and the CFL step kept on the device.  The
state (2.4 GB in the default FP32 perturbation form, 4.8 GB in FP64, for the
512x1024x128 bi-fluid grid) is far larger than L2, so no flush is needed
between steps.  The line also carries the FP64 form's throughput on the same
grid, the FP32 form's relative L1 error against the FP64 form over the timed
workload's 50 steps (and over 100 steps of the 128x256x32 noisy disc), the
roofline of the stage kernel against HBM, instruction issue and the FMA
throughput measured in the same run, and the adjoint's cost.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|fp32]
                  [--workload NAME] [--impl ours|reference]

--impl reference times the CPU oracle (the FP64 restatement of the paper's
step that the tests compare against) on the host cores, on a bounded sample
of the same workload (a reduced grid with the same extents and physics).
Under torchrun each rank runs an independent replica on its own GPU ("replicas
only": the method's grid is not sharded across GPUs here); rank 0 prints one
JSON line.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per GB300 (FP64 vs FP32 at ≤1e-5 L1 err); adjoint/forward cost ratio"
UNIT = "cell-updates/s"
HBM_PEAK_FALLBACK = 6800.0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return HBM_PEAK_FALLBACK, "fallback"


def _profile_values(kernel_tag):
    """Key/value lines of the committed ncu summary of this kernel, if it was
    taken on the current kernel source, else None."""
    import glob
    want = _source_hash(kernel_tag)
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", f"{kernel_tag}__*.txt"))):
        vals = {}
        for line in open(path):
            if "=" in line and not line.startswith("#"):
                k, v = line.split("=", 1)
                vals[k.strip()] = v.split("#")[0].strip()
        if vals.get("source_hash") == want:
            vals["_file"] = os.path.basename(path)
            return vals
    return None


# Issue roof of GB300: 4 warp schedulers per SM, one warp instruction each per
# clock, 152 SMs, at the maximum SM clock (2070 MHz).
ISSUE_PEAK_WARP_INST_S = 4 * 152 * 2070e6


def _traffic(kernel_tag, cells):
    """Per-launch DRAM bytes (read + write) of the stage kernel from a committed
    ncu summary (profiles/<kernel_tag>__<workload>.txt) taken on the current
    kernel source, scaled from the captured grid to `cells` (the stage kernels
    stream the grid once per launch, so traffic grows with the cell count).
    Returns (bytes, summary file name) or (None, None)."""
    import glob
    want = _source_hash(kernel_tag)
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", f"{kernel_tag}__*.txt"))):
        vals = {}
        for line in open(path):
            if "=" in line and not line.startswith("#"):
                k, v = line.split("=", 1)
                vals[k.strip()] = v.split("#")[0].strip()
        if vals.get("source_hash") != want:
            continue
        try:
            return float(vals["dram_bytes_per_launch"]) * cells / float(vals["cells"]), os.path.basename(path)
        except (KeyError, ValueError):
            continue
    return None, None


KERNEL_SOURCES = {  # files that define the kernel and its launcher, and the launch-configuration line's token
    "stage_fp32": (("device_common.cuh", "stage_full.cuh", "stage_pert.cuh", "k_stage_pert_f32.cu"), "P32_TR ="),
    "stage_fp64pert": (("device_common.cuh", "stage_full.cuh", "stage_pert.cuh", "k_stage_pert_f64.cu"), "P32_TR ="),
    "stage_fp64": (("device_common.cuh", "stage_full.cuh", "k_stage_full.cu"), "F64_TR ="),
}


def _source_hash(kernel_tag):
    """Hash of a kernel's code (its headers and launcher) and of its launch
    configuration (the tile / thread-count line of launch.cuh), not of its
    callers."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2207_04252_gb300", "csrc")
    files, token = KERNEL_SOURCES[kernel_tag]
    for name in files:
        h.update(open(os.path.join(csrc, name), "rb").read())
    for line in open(os.path.join(csrc, "launch.cuh")):
        if token in line:
            h.update(line.encode())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, device_id):
        self.device_id = device_id
        self.proc = None
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.device_id)],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None:
            return None
        self.out.flush()
        rows = [l.strip().split(",") for l in open(self.out.name) if l.count(",") >= 8]
        os.unlink(self.out.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        reasons = sorted({name for r in rows for name, v in zip(self.REASONS, r[5:9]) if "Active" in v
                          and "Not" not in v})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _gpu_smi_id(torch):
    try:
        uuid = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        return uuid if uuid.startswith("GPU-") else f"GPU-{uuid}"
    except Exception:
        return os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]


def _oracle_sample(name, shape, steps, barrier_at):
    """One process's share of the CPU baseline: `steps` oracle steps of the
    workload on a reduced grid; returns (start, end) wall-clock times."""
    import oracle
    import synthetic as syn
    ws = syn.scaled(syn.by_name(name), *shape, steps=steps)
    o = oracle.Oracle(ws)
    E = oracle.initial_state(o)
    while time.time() < barrier_at:  # start together
        time.sleep(0.001)
    t0 = time.time()
    o.run(E, steps=steps)
    return t0, time.time()


def cpu_baseline(w, steps=7, shape=(64, 128, 32), procs=None):
    """Times the CPU oracle, as it stands, on a bounded sample of the workload:
    the same workload on a reduced grid (same extents and physics), one
    single-threaded oracle process per host core, all started together (the
    oracle itself is serial; the processes are spawned, never forked from this
    CUDA process); about ten seconds of work per process."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    import synthetic as syn
    procs = procs or os.cpu_count() or 1
    ws = syn.scaled(w, *shape, steps=steps)
    with ProcessPoolExecutor(max_workers=procs, mp_context=mp.get_context("spawn")) as ex:
        start_at = time.time() + 5.0 + 0.2 * procs  # past every worker's start-up
        spans = list(ex.map(_oracle_sample, [w.name] * procs, [shape] * procs, [steps] * procs,
                            [start_at] * procs))
    wall = max(e for _, e in spans) - min(b for b, _ in spans)
    return {"value": procs * ws.ncell * steps / wall, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"{steps} RK2 steps of {ws.name} ({ws.ncell} cells, same extents and physics as the "
                      f"timed workload) in each of {procs} single-threaded oracle processes, one per host core",
            "per_process_value": ws.ncell * steps / statistics.median(e - b for b, e in spans)}


def run_reference(args):
    """The reference arm: the CPU oracle on bounded samples of the workload,
    one single-threaded oracle process per host core (as cpu_baseline)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    import synthetic as syn
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = syn.by_name(args.workload)
    shape = (48, 96, 32)
    procs = os.cpu_count() or 1
    ws = syn.scaled(w, *shape, steps=args.steps)
    with ProcessPoolExecutor(max_workers=procs, mp_context=mp.get_context("spawn")) as ex:
        start_at = time.time() + 5.0 + 0.2 * procs
        spans = list(ex.map(_oracle_sample_timed, [w.name] * procs, [shape] * procs, [args.warmup] * procs,
                            [args.steps] * procs, [start_at] * procs))
    el = max(e for _, e in spans) - min(b for b, _ in spans)
    value = procs * ws.ncell * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": w.name, "sample_grid": f"{shape[0]}x{shape[1]}x{shape[2]}",
                       "precision": "fp64"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                             "sample": f"{args.steps} RK2 steps of {ws.name} per timed run in each of {procs} "
                                       f"single-threaded oracle processes, one per host core"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _oracle_sample_timed(name, shape, warmup, steps, barrier_at):
    """A reference-arm process: `warmup` untimed then `steps` timed oracle
    steps of the workload on a reduced grid; returns the timed span."""
    import oracle
    import synthetic as syn
    ws = syn.scaled(syn.by_name(name), *shape, steps=steps)
    o = oracle.Oracle(ws)
    E = oracle.initial_state(o)
    E, _, _ = o.run(E, steps=warmup)
    while time.time() < barrier_at:
        time.sleep(0.001)
    t0 = time.time()
    o.run(E, steps=steps)
    return t0, time.time()


def fp32_error_vs_fp64(R, W, syn, torch, w, steps):
    """Relative L1 error per conserved quantity (the dust's summed over
    species) of the FP32 form against the FP64 form (itself within 1e-12 of
    the CPU oracle) after `steps` steps of workload w at its full size, both
    driven by the FP64 form's dt sequence, with the element-wise error (the
    largest difference over the largest departure from equilibrium of the
    quantity) and the count of faces the FP32 solver handed to its FP64
    fallback."""
    import numpy as np
    g64 = W.Grid(w, precision=R.ROSSBI_FP64)
    g32 = W.Grid(w, precision=R.ROSSBI_FP32_PERT)
    a = g64.initial_state()
    b = g32.initial_state()
    dt = g64.cfl_dt(a)
    for _ in range(steps):
        ndt = g64.step(a, dt=dt, want_next_dt=True)
        g32.step(b, dt=dt)
        dt = ndt
    status = g64.take_status() | g32.take_status()
    nfb = R.rossbi_fallback_count(g32.h)
    E0 = g64.equilibrium()
    V = np.zeros(w.nr)
    f = w.x0[0] * (w.x1[0] / w.x0[0]) ** (np.arange(w.nr + 1) / w.nr)
    V[:] = 0.5 * (f[1:] ** 2 - f[:-1] ** 2)
    nd = (g64.nf - 5) // 4
    groups = {"mass": [4], "momentum": [0, 1, 2], "energy": [3]}
    if nd:
        groups["dust_mass"] = [8 + 4 * s for s in range(nd)]
        groups["dust_momentum"] = [5 + 4 * s + c for s in range(nd) for c in range(3)]
    out, el = {}, {}
    for name, fields in groups.items():  # field by field, to hold one FP64 field on the host at a time
        num = den = 0.0
        dmax = emax = 0.0
        for q in fields:
            x64 = a[q].double().cpu().numpy()
            x32 = b[q].double().cpu().numpy()
            if q < 5:
                x32 = x32 + E0[q][:, None, :]
            num += float((V * np.abs(x32 - x64)).sum())
            den += float((V * np.abs(x64)).sum())
            dmax = max(dmax, float(np.abs(x32 - x64).max()))
            emax = max(emax, float(np.abs(x64 - (E0[q][:, None, :] if q < 5 else 0.0)).max()))
        out[name] = num / den
        el[name] = dmax / emax if emax > 0 else dmax
    g64.close()
    g32.close()
    del a, b
    torch.cuda.empty_cache()
    return {"workload": w.name, "steps": steps, "rel_l1": out, "elementwise_over_max_departure": el,
            "fallback_faces": nfb, "faces": steps * 2 * 3 * w.ncell, "bar": 1e-5,
            "status": R.status_string(status)}


def measure_fp64(R, W, w, torch, steps=2, warmup=3):
    g = W.Grid(w, precision=R.ROSSBI_FP64, stream=torch.cuda.current_stream())
    s = g.initial_state()
    g.cfl_dt(s)
    for _ in range(warmup):
        g.step(s, dt=0.0)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(steps):
        g.step(s, dt=0.0)
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / steps
    g.close()
    del s
    torch.cuda.empty_cache()
    return {"value": w.ncell / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps, "warmup": warmup,
            "dtype": "f64"}


def _timed_steps(g, s, torch, steps, warmup):
    """ms per step of `steps` device-paced steps after `warmup` untimed ones."""
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        g.step(s, dt=0.0)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        g.step(s, dt=0.0)
    t1.record(stream)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1) / steps


def measure_indirect(R, g, s, torch, x_ref=0.7, steps=4, warmup=2):
    """The same step with the indirect gravity of Sect. 2.10 switched on
    (a moments kernel and its reduction before each stage: 4 more launches
    per step)."""
    g.set_indirect(x_ref)
    ms = _timed_steps(g, s, torch, steps, warmup)
    ab = g.indirect_moments(s).tolist()
    status = g.take_status()
    g.set_indirect(0.0)
    return {"x_ref": x_ref, "value": g.w.ncell / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "warmup": warmup, "moments_AB": ab, "status": R.status_string(status)}


def measure_damping(R, g, s, torch, zones=(0.625, 1.68, 1.0), steps=4, warmup=2):
    """The same step with the radial wave-killing zones of Sect. 2.4 on
    (no extra launch: a per-cell relaxation in the stage epilogues)."""
    g.set_damping(zones)
    ms = _timed_steps(g, s, torch, steps, warmup)
    status = g.take_status()
    g.set_damping(None)
    return {"zones": list(zones), "value": g.w.ncell / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "steps": steps, "warmup": warmup, "status": R.status_string(status)}


def measure_explosion(R, W, syn, torch, steps=2, warmup=1):
    """The cylindrical explosion of Sect. 4.1 at the paper's 1600 x 3200 polar
    resolution (one z cell), FP64 form, device-paced steps."""
    w = syn.EXPLOSION
    g = W.Grid(w, precision=R.ROSSBI_FP64, stream=torch.cuda.current_stream())
    s = g.initial_state()
    g.cfl_dt(s)
    ms = _timed_steps(g, s, torch, steps, warmup)
    status = g.take_status()
    g.close()
    del s
    torch.cuda.empty_cache()
    return {"workload": w.name, "value": w.ncell / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "warmup": warmup, "dtype": "f64", "status": R.status_string(status),
            "note": "one z cell: the flat 14x30x1 tile (no z halo, no z sweep)"}


def measure_adjoint(R, W, syn, torch, steps=4, warmup=3):
    """Cost of the FP64 discrete adjoint on the adjoint workload (128x256x32,
    bi-fluid): one rossbi_adjoint_step (forward recompute of the step included)
    over one rossbi_step, both timed with CUDA events on the grid's stream; and
    a whole gradient (forward run with checkpoints + backward sweep) over the
    forward run, for 20 steps with checkpoints every 10."""
    from paper_2207_04252_gb300 import adjoint as adj
    w = syn.ADJOINT
    stream = torch.cuda.current_stream()
    g = W.Grid(w, precision=R.ROSSBI_FP64, stream=stream)
    s = g.initial_state()
    dt = g.cfl_dt(s)
    lam = adj.vortex_core_weights(g).cuda().contiguous()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    fwd_state = s.clone()
    t_fwd = timed(lambda: g.step(fwd_state, dt=dt))
    t_adj = timed(lambda: g.adjoint_step(s, dt, lam))
    # whole gradient through 20 steps (forward with checkpoints every 10,
    # recomputation, 20 adjoint steps) over the plain 20-step forward run,
    # both bracketed by CUDA events on the grid's stream (the span includes
    # any time the host takes between launches)
    dts = [dt] * 20

    def span(fn):
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    def run():
        y = s.clone()
        for d in dts:
            g.step(y, dt=d)

    def grad():
        x = s.clone().requires_grad_(True)
        out = adj.run_steps(g, x, dts, every=10)
        (lam * out).sum().backward()

    run()
    grad()  # warm-up of both
    t_run = span(run)
    t_grad = span(grad)
    status = g.take_status()
    g.close()
    return {"workload": w.name, "forward_step_ms": t_fwd, "adjoint_step_ms": t_adj, "ratio": t_adj / t_fwd,
            "gradient_20_steps_ms": t_grad, "forward_20_steps_ms": t_run,
            "gradient_20_steps_over_forward_run": t_grad / t_run,
            "gradient_steps_note": "forward with checkpoints (20 steps) + recomputation (10) + 20 adjoint steps",
            "status": R.status_string(status)}


def reduce_max(value, dist, device="cuda"):
    """Largest of one float per rank (the job's time is its slowest rank's)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(cells_per_rank, steps, world, elapsed_ms):
    """Whole-job cell-updates/s of `world` replicas that each advanced their
    own grid of cells_per_rank cells by `steps` steps in elapsed_ms."""
    return cells_per_rank * steps * world / (elapsed_ms * 1e-3)


def run_ours(args):
    import numpy as np
    import torch

    import synthetic as syn
    from paper_2207_04252_gb300 import build as lib_build
    from paper_2207_04252_gb300 import rossbi as R
    from paper_2207_04252_gb300 import workloads

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
    lib_build.build()
    w = syn.by_name(args.workload)
    if args.recon == "primitive":  # the primitive-departure option instead of the paper's reconstruction
        from dataclasses import replace
        w = replace(w, recon=syn.RECON_PRIMITIVE)
    prec = {"fp64": R.ROSSBI_FP64, "fp32": R.ROSSBI_FP32_PERT}[args.precision]
    stream = torch.cuda.current_stream()
    g = workloads.Grid(w, precision=prec, stream=stream)
    s = g.initial_state()
    elem = s.element_size()
    if args.indirect:
        g.set_indirect(args.indirect)
    g.cfl_dt(s)
    for _ in range(args.warmup):
        g.step(s, dt=0.0)
    torch.cuda.synchronize()
    status = g.take_status()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    sampler = ClockSampler(_gpu_smi_id(torch))
    R.rossbi_profile_enable(g.h, True)
    R.rossbi_profile_read(g.h)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with sampler:
        barrier()
        start.record(stream)
        for _ in range(args.steps):
            g.step(s, dt=0.0)
        end.record(stream)
        barrier()
    elapsed_ms = start.elapsed_time(end)
    stage_ms, stage_launches = R.rossbi_profile_read(g.h)
    R.rossbi_profile_enable(g.h, False)
    status |= g.take_status()
    elapsed_ms = reduce_max(elapsed_ms, dist)
    clocks = sampler.summary()
    value = job_throughput(w.ncell, args.steps, world, elapsed_ms)

    # end to end through the public API with host buffers (copies inside the timed region)
    e2e_steps = max(1, min(args.steps, 3))
    host = torch.empty(g.shape, dtype=g.dtype, pin_memory=True)
    host.copy_(s)
    hnp = host.numpy()
    dt = R.rossbi_step_host(g.h, hnp, dt=0.0, dust=g.dust)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        dt = R.rossbi_step_host(g.h, hnp, dt=dt, dust=g.dust)
    e2e_s = time.perf_counter() - t0
    state_bytes = g.nf * w.ncell * elem
    e2e = {"value": w.ncell * e2e_steps * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
           "d2h_bytes_per_step": state_bytes}

    peak, peak_kind = _peaks()
    avg_launch_s = stage_ms * 1e-3 / max(1, stage_launches)
    bytes_per_launch = 2.5 * g.nf * elem * w.ncell  # 5F field accesses per cell-step, two launches
    achieved = bytes_per_launch / avg_launch_s / 1e9
    kernel_tag = f"stage_{args.precision}"
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "peak_kind": peak_kind, "kernel": kernel_tag,
                "avg_launch_ms": avg_launch_s * 1e3}
    # secondary figure: against the 2F field accesses per cell-step that a
    # temporally fused two-stage tile (4-deep halo) would need
    achieved_2f = 1.0 * g.nf * elem * w.ncell / avg_launch_s / 1e9
    roofline["secondary_2f"] = {"achieved": achieved_2f, "frac": achieved_2f / peak,
                                "bytes_per_cell_step": 2 * g.nf * elem}
    # the committed captures are of the default (conservative) instantiation
    traffic, src = _traffic(kernel_tag, w.ncell) if args.recon == "conservative" else (None, None)
    if traffic is not None:
        roofline["traffic"] = traffic
        roofline["traffic_source"] = src
    # the stage kernels are bound by instruction issue, not by HBM: the same
    # launches against the issue roof, with the warp instructions per cell of
    # the committed ncu capture of this kernel source
    prof = _profile_values(kernel_tag) if args.recon == "conservative" else None
    roofline_issue = None
    if prof is not None and "warp_instructions_per_cell" in prof:
        ipc = float(prof["warp_instructions_per_cell"])
        achieved_i = ipc * w.ncell / avg_launch_s
        roofline_issue = {"bound": "alu", "achieved": achieved_i, "peak": ISSUE_PEAK_WARP_INST_S,
                          "unit": "warp-instructions/s", "frac": achieved_i / ISSUE_PEAK_WARP_INST_S,
                          "warp_instructions_per_cell": ipc, "source": prof["_file"]}
        # the HBM fraction this kernel could reach at 100 % of the issue roof:
        # the 70 % HBM target is beyond an exact Riemann solve per face
        cells_per_s_cap = ISSUE_PEAK_WARP_INST_S / ipc
        roofline["hbm_frac_at_issue_roof"] = cells_per_s_cap * 2.5 * g.nf * elem / 1e9 / peak
    # the ALU roof: the kernel's arithmetic (FLOP per cell-stage of the
    # state's precision, counted by ncu in the committed capture) against the
    # device's FMA throughput measured here
    roofline_alu = None
    if prof is not None and "flop_per_cell" in prof and rank == 0:
        fma_peak = R.rossbi_measure_fma_peak(args.precision == "fp64", torch.cuda.current_stream())
        achieved_f = float(prof["flop_per_cell"]) * w.ncell / avg_launch_s
        roofline_alu = {"bound": "alu", "achieved": achieved_f / 1e12, "peak": fma_peak / 1e12, "unit": "TFLOP/s",
                        "frac": achieved_f / fma_peak, "flop_per_cell": float(prof["flop_per_cell"]),
                        "precision": args.precision, "peak_kind": "measured (FMA chains, this run)",
                        "source": prof["_file"]}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if args.precision == "fp64" else "f32", "data": "synthetic",
                "config": {"workload": w.name, "precision": args.precision, "cells": w.ncell, "fields": g.nf,
                           "state_bytes": state_bytes, "parallelism": f"replicas{world}",
                           "l2": "inputs larger than L2 (no flush needed)", "indirect_x_ref": args.indirect,
                           "recon": args.recon},
                "roofline": roofline, "roofline_issue": roofline_issue, "roofline_alu": roofline_alu, "e2e": e2e,
                "gpu_launches": (7 if args.indirect else 3) * args.steps, "clocks": clocks,
                "status": R.status_string(status)}
        if args.precision == "fp32" and not args.no_extras:
            fp64 = measure_fp64(R, workloads, w, torch)
            line["fp64_form"] = fp64
            line["fp32_over_fp64"] = value / world / fp64["value"]
            # the FP32 form's error on the timed workload itself (its 50-step
            # run), and on the gas-only disc over 100 steps
            line["fp32_error_vs_fp64"] = fp32_error_vs_fp64(R, workloads, syn, torch, w, w.steps)
            line["fp32_error_vs_fp64_disc"] = fp32_error_vs_fp64(R, workloads, syn, torch, syn.DISC_NOISE,
                                                                 syn.DISC_NOISE.steps)
            line["explosion"] = measure_explosion(R, workloads, syn, torch)
        if not args.no_extras and not args.indirect:
            ind = measure_indirect(R, g, s, torch)
            ind["over_plain_step"] = ind["ms_per_step"] / (elapsed_ms / args.steps)
            line["indirect"] = ind
            dmp = measure_damping(R, g, s, torch)
            dmp["over_plain_step"] = dmp["ms_per_step"] / (elapsed_ms / args.steps)
            line["damping"] = dmp
        line["adjoint_over_forward"] = None
        if not args.no_extras:
            a = measure_adjoint(R, workloads, syn, torch)
            line["adjoint"] = a
            line["adjoint_over_forward"] = a["ratio"]
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(w)
        print(json.dumps(line), flush=True)
    g.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", choices=("fp64", "fp32"), default="fp32")
    ap.add_argument("--workload", default="bifluid_two_vortices_512x1024x128")
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64-form and FP32-error side measurements")
    ap.add_argument("--recon", choices=("conservative", "primitive"), default="conservative",
                    help="gas reconstruction: the paper's conservative departures, or the primitive-departure option")
    ap.add_argument("--indirect", type=float, default=0.0,
                    help="X_ref of the indirect gravity (Sect. 2.10) for the timed steps; 0 = off")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="print only the adjoint cost measurement (adjoint workload, FP64)")
    args = ap.parse_args()
    if args.adjoint_only:
        import torch
        import synthetic as syn
        from paper_2207_04252_gb300 import build as lib_build
        from paper_2207_04252_gb300 import rossbi as R
        from paper_2207_04252_gb300 import workloads
        lib_build.build()
        print(json.dumps(measure_adjoint(R, workloads, syn, torch)), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
