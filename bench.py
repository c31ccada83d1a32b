"""Throughput benchmark of the RKDG + CSWENO step on one GB300 (or N, as
independent replicas).

Workload: the Mach-10 double-Mach-reflection set-up of the paper's Example 5
on [0,4]x[0,1], jittered split-square mesh 960x240 (460,800 triangles),
Euler P2 (24 modal DOF per cell), KXRCF detection with C_K = 1, CSWENO
reconstruction of flagged cells, SSP-RK3, CFL 0.1; FP32 bulk arithmetic with
the smoothness-indicator sums, nonlinear weights, troubled-cell test and
positivity check in FP64.  A step is one SSP-RK3 time step (three stages,
each: operator + RK update, detection, reconstruction, write-back) plus the
CFL reduction.

Metric: element-DOF x RK-stage updates per second = cells * 24 * 3 * steps / s.

The timed steps run in the developed flow: the solver first advances, untimed,
from the projected initial condition to --t-start (default t = 0.18 of the
configuration's t = 0.2 for the double Mach reflection, 0.2 of 0.25 for the
ensemble), then takes --warmup untimed steps and times --steps steps.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (a fixed random subset of cells of the full mesh) instead.
"""
from __future__ import annotations

import argparse
import datetime
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2106_06280_gb300 import workloads as W  # noqa: E402

METRIC = "element-DOF x RK-stage updates/s"
UNIT = "DOF-stage/s"
NX, NY, K = 960, 240, 2
NP, NV = 6, 4
WORKLOADS = {
    "dmr": "double Mach reflection, Euler P2, jittered split-square 960x240 (460,800 triangles), KXRCF + CSWENO, SSP-RK3, CFL 0.1",
    "ensemble": "256 independent four-quadrant Riemann problems, Euler P2, jittered split-square meshes of 2k-60k triangles "
                "(4,984,396 triangles in one disconnected mesh), KXRCF + CSWENO, SSP-RK3, CFL 0.1",
}
WORKLOAD = WORKLOADS["dmr"]


def make_problem(name, seed):
    if name == "ensemble":
        return W.riemann_ensemble(256, seed=1000 + 1000 * (seed - 3))
    return W.double_mach(NX, NY, seed=seed)
FALLBACK_HBM_GBS = 6800.0


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rk = int(os.environ.get("RANK", "0"))
    lr = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rk, lr


def replica_seed(rank: int) -> int:
    """Mesh/initial-condition seed of a rank's replica (replicas only: each GPU
    advances its own independent copy of the workload)."""
    return 3 + rank


def max_over_ranks(ms: float, device: str) -> float:
    """The slowest rank's timed-region milliseconds (the only collective)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world_size: int, ms_max: float) -> float:
    """Units processed by all ranks divided by the slowest rank's time."""
    return units_per_rank * world_size / (ms_max * 1e-3)


def stage_bytes_per_cell(fp32: bool) -> float:
    """Algorithmic DRAM bytes of the operator + RK stage kernel per cell,
    averaged over the three stages: read u^(i-1) (S), write u^(i) (S), read u^n
    (S, stages 2 and 3), geometry (4 inverse-Jacobian + 9 scaled-normal words),
    three neighbour indices (12 B), the packed neighbour faces (1 B) and the
    KXRCF precursors written for the detection (7 words in the cell's record,
    3 face means into the neighbours' records).  Neighbour traces are reuse of
    data already counted."""
    s = 4 if fp32 else 8
    S = NP * NV * s
    geo = 13 * s + 12 + 1
    kx = 10 * s
    return (3 * (2 * S + geo + kx) + 2 * S) / 3.0


# FP64 flops of the Euler P2 operator + RK stage per cell (FMA = 2, reciprocal and
# square root = 1), counted from the stage kernel: 7 volume points x 147 (trace
# 40, flux 19, accumulation 88), 12 face points x 199 (two traces 80, local
# Lax-Friedrichs flux 67, accumulation 52), RK update 120, KXRCF record and the
# positivity screen 110
STAGE_FLOPS_PER_CELL_EULER_P2 = 7 * 147 + 12 * 199 + 120 + 110


def stage_flops_per_cell(csw, pb, shape):
    """FP64 flops per cell-stage of the stage kernel a launch shape runs: the
    count above for k_stage; for k_stage_tiles each cell forms its own traces
    and accumulates at its 12 face points, the local Lax-Friedrichs flux is
    evaluated once per face of the tile's face list (4 points each) and a
    neighbour's trace only across faces to other tiles, counted on this mesh."""
    if not shape[2]:
        return float(STAGE_FLOPS_PER_CELL_EULER_P2)
    nbr = csw.host_mesh(pb, 2)["nbr"]
    nc, blk = nbr.shape[1], shape[0]
    cell = np.arange(nc)[None, :]
    inside = (nbr >= 0) & (nbr // blk == cell // blk) & (nbr != cell)
    outer = ((nbr >= 0) & ~inside).sum() / nc
    flux = (inside.sum() / 2 + (nbr >= 0).sum() - inside.sum() + (nbr < 0).sum()) / nc
    return 7 * 147 + 12 * (40 + 52) + 4 * flux * 67 + 4 * outer * 40 + 120 + 110


def read_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for key in ("hbm_gbs", "hbm_GBps", "hbm"):
                if key in d:
                    return float(d[key]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


def kernel_hash():
    h = hashlib.sha256()
    for f in ("operator.cu", "physics.cuh", "common.cuh", "tables.cuh", "rules.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2106_06280_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


# committed ncu summary of the stage kernel, per workload
PROFILE_FILES = {"dmr": "k_stage_euler_p2_dmr.md", "ensemble": "k_stage_euler_p2_ensemble.md"}


def read_traffic(khash, workload="dmr"):
    """DRAM bytes per launch of the stage kernel from the committed ncu summary
    of this workload, if there is one and it was taken on the current kernel
    source (else None)."""
    p = os.path.join(ROOT, "profiles", PROFILE_FILES.get(workload, ""))
    if not os.path.isfile(p):
        return None
    txt = open(p).read()
    m = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", txt)
    t = re.search(r"dram_bytes_per_launch_full_size:\s*([0-9.eE+]+)", txt)
    if not m or not t or m.group(1) != khash:
        return None
    return float(t.group(1))


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples (every 50 ms) around the
    timed region; stop() keeps the samples whose timestamps fall inside the
    host-side window of the timed region (all samples when none do, which the
    result says)."""

    def __init__(self):
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"cswdg_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "50"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, dev, t0=None, t1=None):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        out = parse_clock_samples(self.path, dev, t0, t1)
        try:
            os.remove(self.path)
        except OSError:
            pass
        return out


def parse_clock_samples(path, dev, t0=None, t1=None):
    """Median SM clock, maximum SM clock and the active throttle reasons of
    the nvidia-smi samples of GPU dev in path (timestamp, index, clocks.sm,
    clocks.max.sm, power, reasons.active, hw_slowdown, hw_thermal_slowdown,
    sw_thermal_slowdown, sw_power_cap); the samples timestamped in [t0, t1]
    (host epoch seconds) when there are any, else all of them."""
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    rows = []
    for line in open(path):
        f = [x.strip() for x in line.split(",")]
        if len(f) < 10 or f[1] != str(dev):
            continue
        try:
            ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            ts = None
        try:
            rows.append((ts, float(f[2]), float(f[3]), [n for n, v in zip(names, f[6:10]) if v.lower() == "active"]))
        except ValueError:
            continue
    inside = [r for r in rows if r[0] is not None and t0 is not None and t0 <= r[0] <= t1]
    use = inside if inside else rows
    if not use:
        return None
    return {"sm_mhz": float(np.median([r[1] for r in use])), "sm_max_mhz": float(max(r[2] for r in use)),
            "reasons": sorted({n for r in use for n in r[3]}), "samples": len(use),
            "window": "timed region" if inside else "around the timed region"}


T_START = {"dmr": 0.18, "ensemble": 0.2}
PRECISION_TEXT = {
    "fp32_bulk": "FP32-bulk mode: FP32 state, operator, RK update and reconstruction polynomials; FP64 "
                 "smoothness-indicator sums, beta_1, tau and nonlinear weights; KXRCF and positivity "
                 "decisions screened in FP32, close calls in FP64",
    "fp32": "FP32 mode: as FP32-bulk with the smoothness indicators and weights in float as well",
    "fp64": "FP64 mode: every step in double",
}


def flow_stats(modes, area, gamma=W.GAMMA):
    """Smallest cell-mean density and pressure of a state (user layout)."""
    m = modes[:, :, 0] / np.sqrt(area)[:, None]
    p = (gamma - 1.0) * (m[:, 3] - 0.5 * (m[:, 1] ** 2 + m[:, 2] ** 2) / m[:, 0])
    return {"min_density_mean": float(m[:, 0].min()), "min_pressure_mean": float(p.min()),
            "finite": bool(np.all(np.isfinite(m)))}


def setup_solver(csw, precision, stream, seed=3, workload="dmr", shape=None):
    """Mesh, initial condition (projected, every cell reconstructed once) and
    the stage kernel's launch shape: given, or picked by cswdg_autotune."""
    pb = make_problem(workload, seed)
    s = csw.Solver(csw.EULER, K, precision, csw.LIMITER_KXRCF, c_k=1.0, cfl=0.1, stream=stream)
    s.setup(pb)
    s.project_ic(pb.u0, apply_limiter=2)
    if shape:
        s.set_stage_shape(*shape)
        s.shape = tuple(shape) + (0,) * (3 - len(shape))
    else:
        blk, grid, tile_faces, _ = s.autotune()
        s.shape = (blk, grid, tile_faces)
    return pb, s


def run_ours(args):
    import torch

    ws, rk, lr = dist_info()
    torch.cuda.set_device(lr)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2106_06280_gb300 import build as B
    B.build()
    from paper_2106_06280_gb300 import cswdg as csw

    stream = torch.cuda.current_stream().cuda_stream
    main_prec = {"fp32_bulk": csw.FP32_BULK, "fp32": csw.FP32, "fp64": csw.FP64}[args.precision]
    pb, s = setup_solver(csw, main_prec, stream, seed=replica_seed(rk), workload=args.workload, shape=args.stage_shape)
    shape = s.shape
    nc = pb.mesh.nc
    t_end = pb.t_end
    # timed, warm-up and profiled steps run unclipped (the flow stays valid past the
    # configuration's end time), so every counted step is a full step
    NO_END = 1e300
    area = W.cell_areas(pb.mesh)
    # untimed advance to the developed flow, then the warm-up steps
    t_start = min(args.t_start if args.t_start is not None else T_START[args.workload], t_end)
    wa = time.perf_counter()
    t_dev = s.step(0.0, 10 ** 8, t_start)
    torch.cuda.synchronize()
    advance_s = time.perf_counter() - wa
    state_dev = s.read_modes()  # the developed state, shared with the other precision modes
    dev_stats = flow_stats(state_dev, area)
    s.step(0.0, args.warmup, NO_END)
    torch.cuda.synchronize()
    nflag0 = s.num_flagged()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    clocks = ClockSampler()
    if rk == 0:
        clocks.start()
        time.sleep(0.1)  # the sampler is running before the timed region starts
    barrier()
    torch.cuda.synchronize()
    w0 = time.time()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed_steps")  # lets a profiler select the timed launches
    e0.record()
    s.step(0.0, args.steps, NO_END)
    e1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    w1 = time.time()
    clk = clocks.stop(lr, w0, w1) if rk == 0 else None
    if ws > 1:
        ms = max_over_ranks(ms, "cuda")
    value = whole_job_rate(float(nc) * NP * NV * 3 * args.steps, ws, ms)
    nflag = s.num_flagged()
    t_window_end = s.get_time()

    # per-kernel device time (events after every launch, no graph), same state trajectory
    prof, nl = s.profile_step(0.0, args.profile_steps, NO_END)
    stage_ms = prof["stage"] / (3 * args.profile_steps)
    bpc = stage_bytes_per_cell(args.precision != "fp64")
    achieved = nc * bpc / (stage_ms * 1e-3) / 1e9
    peak, peak_src = read_peak()
    khash = kernel_hash()
    traffic = read_traffic(khash, args.workload)

    # end to end: pinned host state in, one step, state out, through the C interface
    # (float host arrays when the state is float: cswdg_write_modes_f32 / read_modes_f32)
    f32_io = args.precision != "fp64"
    hdt = torch.float32 if f32_io else torch.float64
    host_in = torch.empty((nc, NV, NP), dtype=hdt, pin_memory=True).numpy()
    host_out = torch.empty((nc, NV, NP), dtype=hdt, pin_memory=True).numpy()
    (s.read_modes_f32 if f32_io else s.read_modes)(host_in)
    write_fn, read_fn = (s.write_modes_f32, s.read_modes_f32) if f32_io else (s.write_modes, s.read_modes)
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    # warm-up through the same calls (first launches of the layout kernels, the step
    # graph after an external state write), then the timed iterations
    for _ in range(max(3, args.warmup)):
        write_fn(host_in)
        s.step(0.0, 1, NO_END)
        read_fn(host_out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        write_fn(host_in)
        s.step(0.0, 1, NO_END)
        read_fn(host_out)
    t1 = time.perf_counter()
    e2e_value = float(nc) * NP * NV * 3 * e2e_steps * ws / (t1 - t0)
    e2e_bytes = nc * NV * NP * (4 if f32_io else 8)

    launches = s.launches_per_step(True) * args.steps
    s.close()

    def secondary(precision, nsteps, what):
        """The same workload in another precision mode, from the same developed
        state, device-timed like value."""
        if nsteps <= 0:
            return None
        pb2, s2 = setup_solver(csw, precision, stream, seed=replica_seed(rk), workload=args.workload, shape=args.stage_shape)
        s2.write_modes(state_dev)
        s2.set_time(t_dev)
        s2.step(0.0, args.warmup, NO_END)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record()
        s2.step(0.0, nsteps, NO_END)
        f1.record()
        torch.cuda.synchronize()
        ms2 = f0.elapsed_time(f1)
        prof2, _ = s2.profile_step(0.0, max(1, min(args.profile_steps, nsteps)), NO_END)
        s2.close()
        shape2 = s2.shape
        out2 = {"value": float(nc) * NP * NV * 3 * nsteps / (ms2 * 1e-3), "unit": UNIT,
                "ms_per_step": ms2 / nsteps, "steps": nsteps, "precision": what,
                "stage_shape": {"cells_per_block": shape2[0], "grid": shape2[1] or "one block per tile",
                                "kernel": "k_stage_tiles" if shape2[2] else "k_stage"},
                "kernel_ms_per_step": {k: v / max(1, min(args.profile_steps, nsteps)) for k, v in prof2.items()}}
        if precision == csw.FP64 and fp64_peak:
            st_ms = out2["kernel_ms_per_step"]["stage"] / 3.0
            fpc = stage_flops_per_cell(csw, pb2, shape2)
            ach = nc * fpc / (st_ms * 1e-3) / 1e9
            out2["roofline_fp64"] = {"bound": "fp64", "kernel": out2["stage_shape"]["kernel"] + " (FP64 mode)", "achieved": ach,
                                     "peak": fp64_peak, "unit": "GFLOP/s", "frac": ach / fp64_peak,
                                     "flops_per_cell": fpc,
                                     "peak_source": "measured: cswdg_probe_fp64_fma (FP64 FMA chains, CUDA events)"}
        return out2

    def adjoint(nsteps):
        """Hand-written adjoint on the isentropic-vortex workload (periodic
        [0,10]^2, 300x300 split squares = 180,000 triangles, Euler P2,
        FP32-bulk): nsteps fixed-dt steps forward with checkpoints every 20,
        then the reverse sweep, through cswdg_adjoint_steps from host buffers."""
        if nsteps <= 0:
            return None
        pbv = W.isentropic_vortex(300, seed=5, box=(0.0, 10.0, 0.0, 10.0))
        sv = csw.Solver(csw.EULER, K, csw.FP32_BULK, csw.LIMITER_KXRCF, c_k=1.0, cfl=0.1, stream=stream)
        sv.setup(pbv)
        sv.project_ic(pbv.u0, apply_limiter=1)
        u0v = sv.read_modes()
        dtv = 0.5 * sv.cfl_dt()
        gTv = np.zeros_like(u0v)
        gTv[:, 0, :] = 2.0 * u0v[:, 0, :]
        sv.set_time(0.0)
        sv.adjoint_steps(u0v, gTv, dtv, 2, 20)  # warm-up (graph capture, allocations)
        sv.set_time(0.0)
        torch.cuda.synchronize()
        ta = time.perf_counter()
        sv.adjoint_steps(u0v, gTv, dtv, nsteps, 20)
        tb = time.perf_counter()
        ncv = pbv.mesh.nc
        sv.close()
        return {"workload": "isentropic vortex, periodic [0,10]^2, 180,000 triangles, Euler P2, FP32-bulk, fixed dt",
                "steps": nsteps, "checkpoint_every": 20, "seconds": tb - ta,
                "value": float(ncv) * NP * NV * 3 * nsteps / (tb - ta), "unit": UNIT,
                "note": "forward with checkpoints + recomputation + reverse sweep, host buffers in and out; "
                        "value counts the forward DOF-stage updates once"}

    def l1_vs_fp64(nsteps):
        """FP32-bulk against FP64 on the same GPU: both from the same projected,
        every-cell-limited initial state, nsteps steps of the same fixed dt (half
        the FP64 CFL step) from the developed state, then the area-weighted L1
        difference of the density means relative to the L1 norm of the FP64
        density means."""
        if nsteps <= 0:
            return None
        res = {}
        for name, prec in (("fp64", csw.FP64), ("fp32_bulk", csw.FP32_BULK)):
            pbl, sl = setup_solver(csw, prec, stream, seed=replica_seed(rk), workload=args.workload, shape=args.stage_shape)
            sl.write_modes(state_dev)
            if name == "fp64":
                dtl = 0.5 * sl.cfl_dt()
            sl.set_time(t_dev)
            sl.step(dtl, nsteps, 1e300)
            res[name] = sl.read_modes()[:, 0, 0]
            sl.close()
        rho64, rho32 = res["fp64"] / np.sqrt(area), res["fp32_bulk"] / np.sqrt(area)
        return {"steps": nsteps, "dt": dtl, "quantity": "density cell means", "from_t": t_dev,
                "l1_rel": float(np.sum(area * np.abs(rho32 - rho64)) / np.sum(area * np.abs(rho64)))}

    try:
        fp64_peak = csw.probe_fp64_fma(stream)
    except Exception:
        fp64_peak = None
    adj = adjoint(args.adjoint_steps)
    fp32 = secondary(csw.FP32, args.fp32_steps, "FP32 mode: smoothness indicators and nonlinear weights in float as well "
                                                 "(quotient forms), FP64 only for close calls of the decisions")
    fp64 = secondary(csw.FP64, args.fp64_steps, "FP64 mode: every step in double")

    if rk != 0:
        return None
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "cells": nc, "degree": K, "dof_per_cell": NP * NV,
                   "precision": PRECISION_TEXT[args.precision],
                   "limiter": "KXRCF C_K=1 + CSWENO", "initial_condition": "L2 projection, every cell reconstructed once",
                   "l2": f"inputs larger than L2: per-step working set about {nc * (3 * NP * NV * 4 + 52) / 1e6:.0f} MB "
                         f"(three {nc * NP * NV * 4 / 1e6:.0f} MB state arrays, {nc * 52 / 1e6:.0f} MB geometry, "
                         "operator blocks of flagged cells) > 129 MB L2",
                   "replicas": "one independent copy of the workload per GPU" if ws > 1 else None,
                   "timed_window": {"t_start": t_dev, "t_end": t_window_end,
                                    "untimed_advance": {"from_t": 0.0, "seconds": advance_s},
                                    "flagged_cells_first_pass": nflag0, "flagged_cells_last_pass": nflag,
                                    "flagged_fraction": [nflag0 / nc, nflag / nc]},
                   "state_at_t_start": dev_stats,
                   "stage_shape": {"cells_per_block": shape[0], "grid": shape[1] or "one block per tile",
                                   "kernel": "k_stage_tiles (each face once per tile)" if shape[2] else "k_stage (every cell its three faces)",
                                   "chosen_by": "given" if args.stage_shape else "cswdg_autotune"}},
        "roofline": {"bound": "hbm", "kernel": ("k_stage_tiles" if shape[2] else "k_stage") + " (operator + RK update)", "achieved": achieved, "peak": peak,
                     "peak_source": peak_src, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "bytes_per_cell_algorithmic": bpc, "stage_ms": stage_ms,
                     "kernel_ms_per_step": {k: v / args.profile_steps for k, v in prof.items()}},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": e2e_bytes,
                "d2h_bytes_per_step": e2e_bytes, "steps": e2e_steps,
                "path": ("cswdg_write_modes_f32(pinned host) + cswdg_step + cswdg_read_modes_f32(pinned host)" if f32_io else
                         "cswdg_write_modes(pinned host) + cswdg_step + cswdg_read_modes(pinned host)")},
        "gpu_launches": launches,
        "clocks": clk,
        "adjoint": adj,
        "fp32_bulk_vs_fp64_l1": l1_vs_fp64(args.l1_steps),
        "fp32_weights": fp32,
        "fp64": fp64,
        "fp64_peak_gflops": fp64_peak,
    }
    if args.cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.cpu_sample, workload=args.workload)
    return out


def cpu_prepare(sample, seed=3, workload="dmr"):
    """The FP64 oracle on a fixed random sample of the cells of the same mesh
    and initial state: the sample, its two-cell neighbourhood projected and
    its neighbours reconstructed once (as the GPU run's initial condition)."""
    import oracle
    pb = make_problem(workload, seed)
    o = oracle.Oracle(pb, k=K, limiter=1)
    oa = oracle.Oracle(pb, k=K, limiter=2)
    rng = np.random.default_rng(12345)
    cells = np.sort(rng.choice(pb.mesh.nc, size=sample, replace=False)).astype(np.int32)
    nb, _, _ = o.connectivity()
    near = np.unique(np.concatenate([cells, nb[cells].ravel()]))
    near = near[near >= 0]
    nb2 = nb[near].ravel()
    near2 = np.unique(np.concatenate([near, nb2[nb2 >= 0]])).astype(np.int32)
    u = np.zeros((pb.mesh.nc, NV, NP))
    o.project_cells(pb.u0, near2, u)
    lim, _ = oa.limit_cells(u, near)
    u[near] = lim
    return {"o": o, "u": u, "cells": cells, "nc": pb.mesh.nc}


def cpu_time(prep, n):
    """One SSP-RK3 step's work of the oracle, single thread, on the first n
    sample cells: 3 x (operator + KXRCF on them + reconstruction of the flagged
    ones).  Returns (seconds, flagged cells per stage)."""
    o, u, cells = prep["o"], prep["u"], prep["cells"][:n]
    t0 = time.perf_counter()
    nflag = 0
    for _ in range(3):
        o.rhs_cells(u, cells)
        fl, _ = o.detect_cells(u, cells)
        flagged = cells[fl.astype(bool)]
        nflag += len(flagged)
        if len(flagged):
            o.limit_cells(u, flagged)
    return time.perf_counter() - t0, nflag // 3


def cpu_baseline(sample, seed=3, workload="dmr"):
    """The FP64 oracle as it stands, single thread, on a fixed random sample of
    the cells of the same mesh and initial state: one SSP-RK3 step's work on
    the sample = 3 x (operator on the sample + KXRCF on the sample +
    reconstruction of the flagged sample cells)."""
    prep = cpu_prepare(sample, seed, workload)
    dt, nflag = cpu_time(prep, sample)
    return {"value": sample * NP * NV * 3 / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{sample} random cells of the {prep['nc']:,}-cell mesh at the initial state, one SSP-RK3 step's work "
                      f"(3 x operator + KXRCF on the sample, CSWENO on its flagged cells: {nflag} per stage); "
                      f"{dt:.1f} s",
            "seconds": dt}


def run_reference(args):
    ws, rk, lr = dist_info()
    if rk != 0:
        return None
    # each step times one SSP-RK3 step's work on a sample of the cells; the
    # sample shrinks with the step count so that the whole run stays bounded
    # (about 20 steps' worth of --ref-sample cells, at least 100 cells a step)
    nsteps = max(1, args.steps)
    n = max(100, min(args.ref_sample, (20 * args.ref_sample) // nsteps))
    prep = cpu_prepare(args.ref_sample, workload=args.workload)
    for _ in range(args.warmup):
        cpu_time(prep, min(n, 100))
    vals = []
    t0 = time.perf_counter()
    nflag = 0
    for _ in range(nsteps):
        dt, nflag = cpu_time(prep, n)
        vals.append(n * NP * NV * 3 / dt)
    t1 = time.perf_counter()
    cb = {"sample": f"{n} random cells of the {prep['nc']:,}-cell mesh per step (one SSP-RK3 step's work: 3 x operator + "
                    f"KXRCF on the sample, CSWENO on its flagged cells, {nflag} in the last stage), median over "
                    f"{nsteps} steps"}
    value = float(np.median(vals))
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * (t1 - t0) / nsteps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOADS[args.workload], "degree": K},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": cb["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default="fp32_bulk", choices=["fp32_bulk", "fp32", "fp64"],
                    help="precision mode of the timed leg (the others are reported beside it)")
    ap.add_argument("--t-start", type=float, default=None,
                    help="untimed advance to this time before the warm-up (default: dmr 0.18, ensemble 0.2)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dmr", choices=sorted(WORKLOADS))
    ap.add_argument("--profile-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--fp64-steps", type=int, default=100)
    ap.add_argument("--fp32-steps", type=int, default=2000)
    ap.add_argument("--adjoint-steps", type=int, default=100)
    ap.add_argument("--l1-steps", type=int, default=20)
    ap.add_argument("--stage-shape", type=lambda v: tuple(int(x) for x in v.split(",")), default=None,
                    help="cells per block, grid and tile_faces 0/1 of the stage kernel (e.g. 256,304,1); default: autotune")
    ap.add_argument("--cpu-sample", type=int, default=200000)
    ap.add_argument("--ref-sample", type=int, default=4000)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    args = ap.parse_args()
    out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
