#!/usr/bin/env python3
"""Benchmark of the asynchronous compressible-flow hot path on GB300.

Workload (one "step" = one full time step of the method: 5 LSERK4 stages, each a fused
RHS + AT-halo + stage update over all sub-domains, then the three tenth-order filter passes):
3-D Taylor-Green vortex, Navier-Stokes, Re 1600, Mach 0.1, gamma 1.4, Pr 0.71, periodic
[0, 2 pi]^3 at 128^3, FP64, 4 x 4 x 4 = 64 sub-domains of 32^3, SAA with seeded uniform delays
0..3 per face per step (AT4 schemes), after the 5 synchronous warm-up steps.

Metric: point-RK-stage updates per second (Mpoint-stage/s) = 128^3 x 5 x steps / time.

  value     device-resident, CUDA events on the solver's stream around K steps (barrier and
            synchronize on both sides, max over ranks); the working set (~1.8 GB) is larger
            than the 129 MB L2.
  e2e       the same metric through the public API with host buffers: per step the state is
            copied in from pinned host memory, stepped, and copied back out; host_link gives the
            measured bandwidth of those copies and the floor they put under an e2e step.
  roofline  the dominant kernel's achieved FP64 rate (algorithmic flops per launch / average
            event-timed launch duration) against the GB300 FP64 peak.
  cpu_baseline  the FP64 CPU oracle on the host cores on a bounded sample of the workload.

forms (same metric, one GPU; each a dict in the JSON line):
  fp32_intermediates, fp32_intermediates_256   the precision form (FP32 derivative / flux / filter
            intermediates, FP64 state and AT application) at 128^3 and at 256^3 with CAA L = 4,
            with its error against the FP64 path;
  batched_blocks[_curvilinear][_fp32_intermediates]   12 independent periodic blocks of the
            airfoil grid's uneven sizes (20.8 M points) in one context, CUDA graph, autotuned;
  cgrid_naca0012[_fp32_intermediates]   the connected 12-block NACA0012 C-grid (22.0 M points:
            wake cut, walls, far field, outflows, spanwise interpolation), SAA 0..2, CUDA graph;
  learned_halo   the learned stage-0 halo against the plain AT extrapolation;
  algorithms     SA, CAA and SAA with the fourth- and second-order schemes on the 128^3 grid.

--impl reference times the oracle itself (the CPU program the GPU path is checked against) on
the same configuration and metric; under torchrun only rank 0 runs it.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Mpoint-RK-stage updates/s and % HBM peak; forms vs plain FP64 at stated L2 error"
UNIT = "Mpoint-stage/s"
SM_COUNT = 152
FP64_FLOP_PER_CLK_SM = 4        # 2 FP64 FMA per clock per SM on GB300
HBM_GBS_FALLBACK = 6800.0

# ncu dram__bytes_read.sum + dram__bytes_write.sum per launch of each kernel kind, with the sha1 of
# the flux kernel's source they were taken from (kernels_sha1; null once it changes); filled
# from profiles/.
TRAFFIC = {"source_sha1": "c488e6aad06093ada1bf5e2b117f15b1ca3752b9",
           # k_flux<double,3>: 92.56 MB read + 81.52 MB written per launch in an ncu capture of the
           # 96^3 case (27 sub-domains of 32^3), x 64/27 for the 64 sub-domains of 128^3
           "bytes_per_launch": {"flux": 412.6e6}}


def kernels_sha1(root: str = ROOT) -> str:
    """sha1 of the source the flux kernel is built from: its section of kernels.cu (from the k_flux
    banner to the k_rk banner), the device helpers it includes, and the descriptors it reads
    (Geometry, Physics, SubDev); other kernels' edits leave it unchanged."""
    csrc = os.path.join(root, "paper_2506_03027_gb300", "csrc")
    with open(os.path.join(csrc, "kernels.cu")) as f:
        k = f.read()
    a = k.index("// " + "-" * 79 + " k_flux")
    b = k.index("// " + "-" * 79 + " k_rk")
    with open(os.path.join(csrc, "device_common.cuh")) as f:
        dc = f.read()
    with open(os.path.join(csrc, "cfs_internal.h")) as f:
        h = f.read()
    structs = "".join(h[h.index("struct " + n + " {"):h.index("};", h.index("struct " + n + " {")) + 2]
                      for n in ("SubDev", "Geometry", "Physics"))
    return hashlib.sha1((k[a:b] + dc + structs).encode()).hexdigest()


def host_link(host, nbytes: int) -> dict:
    """Bandwidth of the host link for the e2e copies: the pinned state buffer to a device buffer
    and back (copy engine, CUDA events, median of 5 after 2 warm-ups), and the floor they put
    under an e2e step (one copy each way per step)."""
    import torch
    dev = torch.empty_like(host, device="cuda")
    st = torch.cuda.current_stream()
    out = {}
    for name, dst, src in (("h2d", dev, host), ("d2h", host, dev)):
        ts = []
        for rep in range(7):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            dst.copy_(src, non_blocking=True)
            e1.record(st)
            e1.synchronize()
            if rep >= 2:
                ts.append(e0.elapsed_time(e1))
        out[name + "_gbs"] = nbytes / (sorted(ts)[len(ts) // 2] * 1e-3) / 1e9
    out["copy_floor_ms_per_step"] = (nbytes / out["h2d_gbs"] + nbytes / out["d2h_gbs"]) / 1e6
    del dev
    return out


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The largest value of a per-rank number (a time) over the ranks of the process group; the
    number itself on a single rank."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput in millions per second: the units all ranks processed over the time
    of the slowest rank (replicas: every rank advances its own problem of the same size)."""
    return units_per_rank * world / seconds / 1e6


def workload(algo="SAA", grid=128, split=4):
    from paper_2506_03027_gb300 import inputs as I
    c = I.tgv_case(grid, split, algo)
    # Asynchronous runs need a smaller step for stability.  Measured at 128^3 on 32^3
    # sub-domains over 600 steps: SAA with delays 0..3 is stable at CFL 0.05 only (non-finite by
    # step 75/100/175 at CFL 0.5/0.25/0.1), CAA L = 4 at CFL <= 0.25, SA at 0.5.  The paper cut
    # the step 10x for its asynchronous TGV runs.  The cost of a step does not depend on dt.
    cfl = {"SA": 0.5, "CAA": 0.25, "SAA": 0.05}[algo]
    c = c.replace(dt=I.cfl_dt(c, I.tgv_state(c), cfl))
    return c


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def rel_l2(a, ref):
    """Relative L2 difference per conserved variable: rho and rho E against their own norms, the
    momentum components against the norm of the momentum vector field."""
    mom = math.sqrt(sum(float(np.linalg.norm(ref[v])) ** 2 for v in (1, 2, 3)))
    return [float(np.linalg.norm(a[v] - ref[v])) / (mom if v in (1, 2, 3) else float(np.linalg.norm(ref[v])))
            for v in range(5)]


def rel_l2_own(a, ref):
    """The same with every variable against its own norm."""
    return [float(np.linalg.norm(a[v] - ref[v]) / np.linalg.norm(ref[v])) for v in range(5)]


def face_points(case, depth):
    """Points of the face strips (depth `depth`) of all sub-domains along each axis."""
    from paper_2506_03027_gb300 import inputs as I  # noqa: F401
    tot = 0
    for ix in range(case.px):
        sx = case.nx // case.px + (1 if ix < case.nx % case.px else 0)
        for iy in range(case.py):
            sy = case.ny // case.py + (1 if iy < case.ny % case.py else 0)
            for iz in range(case.pz):
                sz = case.nz // case.pz + (1 if iz < case.nz % case.pz else 0)
                tot += 2 * depth * (sy * sz + sx * sz + sx * sy)
    return tot


def algorithmic_flops(case, kind):
    """FP64 flops per launch that the method needs in each kernel (FMA = 2 flops), counted from
    the operations of the 3-D Navier-Stokes CD4 path; see the design notes for the breakdown."""
    N = case.npts
    r = 2 if case.order == 4 else 1
    if kind == "flux":
        # owned points: 12 CD gradients (5 flops each) + divergence (2) + per direction 33 flops of
        # fluxes; strip points beyond a face (depth <= r): the 8 gradients the flux along that axis
        # needs, the divergence and one direction
        return N * (60 + 2 + 3 * 33) + face_points(case, r) * (40 + 2 + 33)
    if kind == "stage_update":
        # 15 CD derivatives (5 flops) + 3 adds per variable, then Q and U updates (5 per variable)
        return N * (5 * (15 + 3) + 5 * 5)
    if kind == "view":
        g = 2 * r
        halo = face_points(case, g) + 0  # face halos; edges and AT weights counted in the notes
        return (N + halo) * 16 + halo * 5 * case.levels * 2
    if kind == "filter":
        return N * 5 * 21
    return 0


def algorithmic_bytes_per_step(case):
    """HBM bytes the method must move per step: state and LSERK register traffic (FP64) of the
    5 stages (120 + 3 x 160 + 120 B per point), the filter passes (read + write, 80 B per point
    per pass) and the ring levels the AT halos read once per stage (C levels x 40 B per halo
    point)."""
    N = case.npts
    r = 2 if case.order == 4 else 1
    g = 2 * r if case.viscous else r
    halo = face_points(case, g)
    stage = N * (120 + 160 * (case.stages - 2) + 120)
    filt = N * 80 * (3 if case.nz > 1 else 2) if case.filter else 0
    ring = halo * case.levels * 40 * case.stages
    return stage + filt + ring


def fused_roofline(case, ktimes):
    """HBM roofline of the fused FP32-intermediate stage kernel (one launch per RK stage):
    algorithmic bytes per launch = the FP64 state and LSERK register traffic (144 B per point,
    averaged over the 5 stages) plus the FP32 halo primitives it reads from the per-step halo
    store (7 x 4 B per face-halo point), over the event-timed average launch."""
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", HBM_GBS_FALLBACK)
    t, n = ktimes.get("stage_update", (0.0, 0))
    if not n:
        return None
    per_launch_s = t / n * 1e-3
    bytes_ = case.npts * (120 + 160 * (case.stages - 2) + 120) / case.stages + face_points(case, 4) * 28
    achieved = bytes_ / per_launch_s / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "bytes_per_launch": bytes_, "ms_per_launch": t / n,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in peaks else "fallback"}


def fp64_peak(local_rank: int = 0):
    """The FP64 pipe rate of this GPU, measured: the library's probe kernel (8 independent DFMA
    chains per thread, 8 CTAs of 256 threads per SM) timed with CUDA events, median of 5 launches
    after a warm-up launch.  Returns TFLOP/s (FMA = 2 flops) and the clock samples taken meanwhile."""
    import torch
    from paper_2506_03027_gb300 import cfs
    blocks, iters = SM_COUNT * 8, 4096
    sink = torch.empty(blocks * 256, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    cfs.cfs_fp64_probe(sink, blocks, iters, st.cuda_stream)
    ts = []
    with ClockSampler(local_rank) as clk:
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            cfs.cfs_fp64_probe(sink, blocks, iters, st.cuda_stream)
            e1.record(st)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
    ms = statistics.median(ts)
    fmas = blocks * 256 * iters * 8
    return {"tflops": 2 * fmas / (ms * 1e-3) / 1e12, "ms": ms, "fmas": fmas,
            "sm_mhz": clk.summary().get("sm_mhz")}


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2506_03027_gb300 import build as B
    from paper_2506_03027_gb300 import cfs
    from paper_2506_03027_gb300 import inputs as I

    torch.cuda.set_device(local_rank)
    if rank == 0:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    B.build()
    case = workload(args.schedule, args.grid, args.split)
    case = case.replace(seed=case.seed + rank)
    K, W = args.steps, args.warmup
    total = W + 3 * K + 8  # warm-up, timed steps, the per-kernel timing pass, end-to-end steps
    delays = I.saa_delays(case, total)
    U0 = I.tgv_state(case)
    stream = torch.cuda.current_stream()

    tiles = tuple(int(t) for t in args.tiles.split(",")) if args.tiles else None
    # the step is captured once in a CUDA graph and replayed (the step index lives on the device)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    solver = cfs.Solver(case, precision=args.precision, tiles=tiles, stream=stream, graph=True)
    solver.set_schedule(delays=delays)
    solver.set_state(U0)
    solver.step(W)
    torch.cuda.synchronize()

    # ---------------- device-resident timed region (graph replays, no per-kernel events)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        e0.record(stream)
        solver.step(K)
        e1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    launches = solver.launches()
    ms = max_over_ranks(ms, world)
    n_units = case.npts * case.stages * K * world
    value = whole_job_rate(case.npts * case.stages * K, world, ms * 1e-3)

    # ---------------- per-kernel times: a separate pass of K steps with CUDA events around every
    # launch on the solver's stream (this bypasses the graph; not part of the timed value)
    cfs.cfs_set_timing(solver.ctx, True)
    solver.step(K)
    ktimes = cfs.cfs_get_timing(solver.ctx)
    cfs.cfs_set_timing(solver.ctx, False)
    torch.cuda.synchronize()

    # ---------------- end to end through the public API with host buffers
    host = torch.empty((5, case.nz, case.ny, case.nx), dtype=torch.float64, pin_memory=True)
    hnp = host.numpy()
    solver.get_state(hnp)
    Ke = max(3, K // 2)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(Ke):
        solver.set_state(hnp)          # host -> device copy of the step's input
        solver.step(1)
        solver.get_state(hnp)          # device -> host copy of the step's result (synchronises)
    torch.cuda.synchronize()
    te = time.perf_counter() - t0
    te = max_over_ranks(te, world)
    e2e_value = whole_job_rate(case.npts * case.stages * Ke, world, te)
    state_bytes = 5 * case.npts * 8
    link = host_link(host, state_bytes)
    U_fp64 = solver.get_state()
    n_done = solver.n
    solver.close()
    torch.cuda.set_stream(torch.cuda.default_stream())
    stream = torch.cuda.current_stream()

    # ---------------- precision form (FP32 intermediates), same steps, error vs the FP64 path
    forms = None
    if args.precision == 0 and not args.no_forms:
        from paper_2506_03027_gb300 import autotune
        tiles32 = autotune.tune(case, precision=1, use_cache=False)
        s32 = cfs.Solver(case, precision=1, tiles=tiles32)
        s32.set_schedule(delays=delays)
        s32.set_state(U0)
        s32.step(W)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        cfs.cfs_set_timing(s32.ctx, True)
        f0.record(stream)
        s32.step(K)
        f1.record(stream)
        torch.cuda.synchronize()
        ms32 = f0.elapsed_time(f1)
        kt32 = cfs.cfs_get_timing(s32.ctx)
        cfs.cfs_set_timing(s32.ctx, False)
        s32.step(n_done - s32.n)
        U32 = s32.get_state()
        s32.close()
        err = rel_l2(U32, U_fp64)
        err_own = rel_l2_own(U32, U_fp64)
        forms = {"fp32_intermediates": {"value": n_units / (ms32 * 1e-3) / 1e6, "unit": UNIT,
                                        "speedup_vs_fp64": ms / ms32,
                                        "rel_l2_vs_fp64_path": err, "rel_l2_own_norm_vs_fp64_path": err_own,
                                        "after_steps": n_done,
                                        "tiles_autotuned": list(tiles32),
                                        "per_kernel_ms": {k: round(v[0] / max(v[1], 1), 4) for k, v in kt32.items() if v[1]},
                                        "fused_stage_roofline": fused_roofline(case, kt32)}}

    if args.precision == 0 and not args.no_forms and world == 1:
        forms["fp32_intermediates_256"] = precision_form_256(args)

    # ---------------- batched uneven blocks (one launch per kernel over all blocks, CUDA graph)
    if args.precision == 0 and not args.no_forms and world == 1:
        forms = forms or {}
        forms["batched_blocks"] = batched_form(args, 0)
        forms["batched_blocks_fp32_intermediates"] = batched_form(args, 1)
        forms["batched_blocks_curvilinear"] = batched_form(args, 0, curvilinear=True)
        forms["batched_blocks_curvilinear_fp32_intermediates"] = batched_form(args, 1, curvilinear=True)
        forms["cgrid_naca0012"] = cgrid_form(args, 0)
        forms["cgrid_naca0012_fp32_intermediates"] = cgrid_form(args, 1)

    # ---------------- learned halo predictor (trained here on synchronous-run halos)
    if args.precision == 0 and not args.no_forms and not args.no_learned and world == 1:
        forms = forms or {}
        forms["learned_halo"] = learned_form(args)

    # ---------------- the three algorithms and the second-order schemes on the same grid
    if args.precision == 0 and not args.no_forms and world == 1:
        forms = forms or {}
        forms["algorithms"] = algorithms_form(args)
        forms["compact_euler"] = compact_form(args)
        forms["static_diagnostics"] = static_diagnostics_form()

    # ---------------- roofline of the dominant kernel
    peaks = measured_peaks()
    clocks = clk.summary()
    sm_max = clocks.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    kinds = {k: v for k, v in ktimes.items() if v[1] > 0 and k != "diagnostics"}
    dom = max(kinds, key=lambda k: kinds[k][0])
    dom_ms, dom_n = kinds[dom]
    flops = algorithmic_flops(case, dom)
    achieved_tf = flops / (dom_ms / dom_n * 1e-3) / 1e12
    if args.precision == 0:
        probe = fp64_peak(local_rank)
        peak_tf = probe["tflops"]
        roof = {"bound": "alu", "achieved": achieved_tf, "peak": peak_tf, "unit": "TFLOP/s",
                "frac": achieved_tf / peak_tf, "kernel": dom,
                "peak_source": "measured FP64 pipe rate (cfs_fp64_probe: dependent-free DFMA chains, median of 5, "
                               "on this GPU in this run)",
                "fp64_probe": probe,
                "nominal_peak": SM_COUNT * FP64_FLOP_PER_CLK_SM * sm_max * 1e6 / 1e12}
    else:
        # the FP32-intermediate form's dominant kernel: the fused stage against HBM
        roof = fused_roofline(case, ktimes) or {"bound": "hbm", "achieved": None, "peak": None, "unit": "GB/s",
                                                "frac": None}
        roof["kernel"] = dom
    tr = TRAFFIC["bytes_per_launch"].get(dom) if TRAFFIC["source_sha1"] == kernels_sha1() else None
    roof["traffic"] = tr
    roof["per_kernel_ms"] = {k: round(v[0] / max(v[1], 1), 4) for k, v in kinds.items()}
    hbm = peaks.get("hbm_gbs", HBM_GBS_FALLBACK)
    step_bytes = algorithmic_bytes_per_step(case)
    hbm_frac = step_bytes * K / (ms * 1e-3) / 1e9 / hbm

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == 0 else "f64-state/f32-intermediates", "data": "synthetic",
        "config": {"workload": f"Taylor-Green vortex NS {case.nx}^3, {case.px}x{case.py}x{case.pz} sub-domains, {args.schedule}-AT "
                               "delays 0..3 per face per step, LSERK4-CD4-AT4, 10th-order filter alpha_f 0.499",
                   "grid": [case.nx, case.ny, case.nz], "subdomains": case.nsub, "schedule": args.schedule,
                   "precision": "fp64" if args.precision == 0 else "fp32-intermediates",
                   "l2_policy": "working set larger than L2 (no flush needed)",
                   "replicas": "independent problem per rank" if world > 1 else None},
        "hbm_frac_algorithmic": hbm_frac,
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
                "d2h_bytes_per_step": state_bytes, "ms_per_step": te * 1e3 / Ke, "host_link": link},
        "gpu_launches": launches,
        "launches_per_step": launches / K,
        "cuda_graph": True,
        "clocks": clocks,
    }
    if forms:
        line["forms"] = forms
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(case)
    return line


NACA_BLOCKS = [(512, 192, 64), (384, 192, 64), (256, 192, 64), (256, 128, 64), (192, 128, 64), (128, 128, 64),
               (192, 96, 32), (128, 96, 32), (96, 96, 32), (128, 64, 32), (96, 64, 32), (96, 64, 32)]


def batched_blocks():
    """Twelve independent periodic blocks with the uneven sizes of a 12-block airfoil C-grid
    (96 x 64 x 32 up to 512 x 192 x 64, 20.8 M points), Navier-Stokes TGV fields, sub-domains of
    about 32-64 points per axis, SAA delays 0..2."""
    from paper_2506_03027_gb300 import inputs as I
    base = I.tgv_case(32, 1, "SAA", kmax=2)
    blocks = []
    for (nx, ny, nz) in NACA_BLOCKS:
        b = base.replace(nx=nx, ny=ny, nz=nz, px=max(1, nx // 64), py=max(1, ny // 64), pz=max(1, nz // 32),
                         lx=2 * math.pi * nx / 128, ly=2 * math.pi * ny / 128, lz=2 * math.pi * nz / 128)
        blocks.append(b)
    dt = min(I.cfl_dt(b, I.tgv_state(b), 0.05) for b in blocks)
    return [b.replace(dt=dt) for b in blocks]


def batched_form(args, precision=0, curvilinear=False):
    """All 12 blocks advance together: every kernel launch covers the sub-domains of all blocks
    (work lists over (block, sub-domain, tile)); the FP32-intermediate form runs one persistent
    fused launch per RK stage (Cartesian blocks).  The step is captured once in a CUDA graph and
    replayed; launch shapes come from the autotuner.  curvilinear: every block on a smoothly
    deformed periodic grid (metric terms of App. A; amplitude 4% of the block's smaller side)."""
    import torch
    from paper_2506_03027_gb300 import autotune
    from paper_2506_03027_gb300 import cfs
    from paper_2506_03027_gb300 import inputs as I
    blocks = batched_blocks()
    if curvilinear:
        blocks = [b.replace(curv=0.04 * min(b.lx, b.ly)) for b in blocks]
    tiles = autotune.tune(blocks[0], precision=precision, blocks=blocks, use_cache=False)
    npts = sum(b.npts for b in blocks)
    nsub = sum(b.nsub for b in blocks)
    K, W = max(3, args.steps // 4), args.warmup
    delays = I.saa_delays(blocks[0].replace(px=nsub, py=1, pz=1), W + K)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        s = cfs.Solver(blocks[0], blocks=blocks, graph=True, stream=st, precision=precision, tiles=tiles)
        s.set_schedule(delays=delays)
        for i, b in enumerate(blocks):
            s.set_state(I.tgv_state(b), block=i)
        s.step(W)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        s.step(K)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        launches = s.launches()
        s.close()
    return {"value": npts * 5 * K / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms / K, "points": npts,
            "blocks": len(blocks), "subdomains": nsub, "cuda_graph": True, "launches_per_step": launches / K,
            "tiles_autotuned": list(tiles),
            "workload": "12 independent periodic NS blocks with the 12-block airfoil C-grid sizes, SAA 0..2, "
                        + ("curvilinear (deformed periodic grids), " if curvilinear else "")
                        + ("FP64" if precision == 0 else
                           "FP32 intermediates (one fused launch per RK stage)")}


def cgrid_form(args, precision=0):
    """The 12-block NACA0012 C-grid (22.0 M points: inner layer 192 x 64 spanwise, outer layer
    64 x 32, segments of 96, 160 and 512 points per side along the C), connected by interfaces
    (the wake cut reversed, inner/outer layers by spanwise interpolation), no-slip walls on the
    airfoil, far field and outflows; Re_c 5e4, M 0.3, SAA delays 0..2 at CFL 0.05 of the smallest
    cell.  All blocks advance in one launch per kernel, the step captured in a CUDA graph, launch
    shapes from the autotuner."""
    import torch
    from paper_2506_03027_gb300 import autotune
    from paper_2506_03027_gb300 import cfs
    from paper_2506_03027_gb300 import inputs as I
    spec = I.CGridSpec()
    if getattr(args, "cgrid_half", False):
        spec = I.CGridSpec(wake=48, aft=80, fore=256, nj_in=96, nj_out=32, nz_in=32, nz_out=16)
    mb = I.naca_cgrid(spec, algo="SAA", kmax=2)
    mb = mb.replace_all(dt=I.cgrid_dt(mb, 0.05))
    U0 = I.cgrid_state(mb, spec)
    if args.only_form and args.tiles:
        tiles = tuple(int(t) for t in args.tiles.split(","))
    else:
        tiles = autotune.tune(mb, precision=precision, use_cache=False, states=U0)
    K, W = max(3, args.steps // 4), args.warmup
    delays = I.saa_delays(mb.case.replace(px=mb.nsub, py=1, pz=1), W + K)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        s = cfs.Solver(mb, graph=True, stream=st, precision=precision, tiles=tiles)
        s.set_schedule(delays=delays)
        s.set_states(U0)
        s.step(W)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        s.step(K)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        launches = s.launches()
        d = s.diagnostics(check_finite=False)
        walls_at_rest = all(bool(np.all(s.get_state(block=b)[1:4, :, 0, :] == 0.0)) for b in range(1, 5))
        s.close()
    return {"value": mb.npts * 5 * K / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms / K, "points": mb.npts,
            "blocks": len(mb.blocks), "subdomains": mb.nsub, "cuda_graph": True,
            "launches_per_step": launches / K, "tiles_autotuned": list(tiles),
            "finite": bool(d[7] == 0.0), "wall_points_at_rest": walls_at_rest, "K_after": float(d[0]),
            "workload": "NACA0012 12-block C-grid (interfaces, wake cut, walls, far field, outflows), NS Re_c 5e4 "
                        "M 0.3, SAA 0..2, " + ("FP64" if precision == 0 else "FP32 intermediates (one fused launch per RK stage)")}


def precision_form_256(args):
    """The precision configuration: TGV 256^3 with 8^3 sub-domains, CAA L = 4 (CFL 0.25), FP32
    derivative/flux/filter intermediates against the FP64 path from the same initial state:
    relative L2 error per conserved variable after `nst` steps, error of the kinetic-energy
    dissipation rate -dK/dt (central differences of the per-step K history), and throughput of
    both paths."""
    import torch
    from paper_2506_03027_gb300 import cfs
    from paper_2506_03027_gb300 import inputs as I
    case = I.tgv_case(256, 8, "CAA")
    case = case.replace(dt=I.cfl_dt(case, I.tgv_state(case), 0.25))
    U0 = I.tgv_state(case)
    nst, K, W = 40, 10, 4
    from paper_2506_03027_gb300 import autotune
    tiles = {0: None, 1: autotune.tune(case, precision=1, use_cache=False)}
    res = {}
    for prec in (0, 1):
        s = cfs.Solver(case, precision=prec, tiles=tiles[prec])
        cfs.cfs_set_timing(s.ctx, True)
        s.set_schedule()
        s.set_state(U0)
        s.step(W)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        s.step(K)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / K
        kt = cfs.cfs_get_timing(s.ctx)
        cfs.cfs_set_timing(s.ctx, False)
        s.set_step(0)
        s.set_state(U0)
        ke = [s.diagnostics()[0]]
        for _ in range(nst):
            s.step(1)
            ke.append(s.diagnostics()[0])
        res[prec] = {"ms": ms, "U": s.get_state(), "K": np.array(ke), "kt": kt}
        s.close()
    U64, U32 = res[0]["U"], res[1]["U"]
    err = rel_l2(U32, U64)
    err_own = rel_l2_own(U32, U64)
    eps64 = -(res[0]["K"][2:] - res[0]["K"][:-2]) / (2 * case.dt)
    eps32 = -(res[1]["K"][2:] - res[1]["K"][:-2]) / (2 * case.dt)
    return {"value": case.npts * 5 / (res[1]["ms"] * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": res[1]["ms"],
            "fp64_path": {"value": case.npts * 5 / (res[0]["ms"] * 1e-3) / 1e6, "ms_per_step": res[0]["ms"]},
            "speedup_vs_fp64": res[0]["ms"] / res[1]["ms"],
            "rel_l2_vs_fp64_path": err, "rel_l2_own_norm_vs_fp64_path": err_own, "after_steps": nst,
            "dissipation_rate_rel_err": float(np.abs(eps32 - eps64).max() / np.abs(eps64).max()),
            "tiles_autotuned": list(tiles[1]),
            "per_kernel_ms": {k: round(v[0] / max(v[1], 1), 4) for k, v in res[1]["kt"].items() if v[1]},
            "fused_stage_roofline": fused_roofline(case, res[1]["kt"]),
            "workload": "TGV NS 256^3, 8x8x8 sub-domains, CAA L=4 AT4 at CFL 0.25, filter alpha_f 0.499; "
                        "error against the FP64 path from the same initial state"}


def algorithms_form(args):
    """Throughput of the synchronous (SA), communication-avoiding (CAA, L = 4) and
    synchronization-avoiding (SAA, delays 0..3) runs of the benchmark grid with the fourth-order
    schemes (Table 1 cases 4 and 6), and of SA / SAA with the second-order ones (cases 1 and 3:
    LSERK2, CD2, AT2).  On one GPU there is no communication for the asynchrony to avoid; this
    measures what the AT halo treatment costs against the synchronous halo."""
    import torch
    from paper_2506_03027_gb300 import cfs
    from paper_2506_03027_gb300 import inputs as I
    K, W = max(3, args.steps // 4), max(args.warmup, 6)
    out = {"unit": UNIT}
    for order in (4, 2):
        for algo in ("SA", "CAA", "SAA"):
            if order == 2 and algo == "CAA":
                continue
            case = workload(algo, 128, 4)
            if order == 2:
                case = case.replace(order=2, kmax=min(case.kmax, 3))
            d = I.saa_delays(case, W + K) if algo == "SAA" else None
            s = cfs.Solver(case)
            try:
                s.set_schedule(delays=d)
                s.set_state(I.tgv_state(case))
                s.step(W)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                s.step(K)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / K
            finally:
                s.close()
            out[f"order{order}_{algo}"] = {"value": case.npts * case.stages / (ms * 1e-3) / 1e6, "ms_per_step": ms}
    out["workload"] = ("TGV NS 128^3, 4x4x4 sub-domains, filter; order 4: LSERK4-CD4-AT4, order 2: LSERK2-CD2-AT2; "
                       "CAA L=4, SAA delays 0..3; steps after the synchronous warm-up")
    return out


def learned_form(args):
    """The learned halo configuration: TGV 256^3 on 8^3 sub-domains of 32^3, SAA with delays 0..4
    at CFL 0.05.  The network is trained on halos of synchronous TGV 128^3 runs taken at the same
    time step (so the level differences it sees have the same size), then SA, plain AT (AT4,
    Eq. 15), the 3-level extrapolation of Eq. 14 alone (the network's base) and the network run
    200 steps from the same initial state on the same delays: each asynchronous run's relative L2
    difference from the synchronous one, and its ms per step.  Beside it the held-out halo errors
    (mean squared, target units) of the 3-level extrapolation, AT4 and the network."""
    from paper_2506_03027_gb300 import inputs as I
    from paper_2506_03027_gb300 import learned as L
    t0 = time.perf_counter()
    big = I.tgv_case(256, 8, "SAA", kmax=4)
    dt = I.cfl_dt(big, I.tgv_state(big), 0.05)
    big = big.replace(dt=dt)
    c = I.tgv_case(128, 4, "SA").replace(dt=dt)
    scales = L.fit_scales(c, seed=1, first_step=9, nsteps=4, per_step=20000)
    X, T = L.generate(c, 9, 40, 20000, seed=2, scales=scales)
    params, hist = L.train(X, T, steps=1500, batch=4096, lr=2e-3, seed=0)
    del X, T
    Xh, Th, A4 = L.generate(c, 60, 66, 20000, seed=3, scales=scales, with_at4=True)
    halo = L.halo_errors(params, Xh, Th, A4)
    del Xh, Th, A4
    train_s = time.perf_counter() - t0
    cmp = L.solver_comparison(big, I.tgv_state(big), params, scales, 200)
    ms = cmp["ms_per_step"]
    return {"rel_l2_vs_sa_after_200_steps": cmp["rel_l2_vs_sa"], "finite": cmp["finite"],
            "ms_per_step": ms, "value_learned": big.npts * 5 / (ms["learned"] * 1e-3) / 1e6,
            "value_at": big.npts * 5 / (ms["AT"] * 1e-3) / 1e6,
            "speedup_vs_plain_at": ms["AT"] / ms["learned"], "unit": UNIT,
            "halo_mse_heldout": halo, "train_loss_first_last": [hist[0][1], hist[-1][1]],
            "train_seconds": train_s, "dt": dt,
            "workload": "TGV NS 256^3, 8^3 sub-domains of 32^3, SAA delays 0..4 at CFL 0.05, 200 steps from t = 0; "
                        "network trained on synchronous TGV 128^3 halos at the same dt; errors against SA, "
                        "momentum components against the momentum vector norm"}


def compact_form(args):
    """The sixth-order compact scheme (Eq. 2, alpha = 1/3) against CD4 on the Euler Taylor-Green
    field: 128^3 on 4^3 sub-domains of 32^3, CAA-AT (L = 4) at CFL 0.25, filter on, CUDA graph;
    ms per step of both and the per-kernel times of the compact path (a separate timing pass)."""
    import torch
    from paper_2506_03027_gb300 import cfs
    from paper_2506_03027_gb300 import inputs as I
    K, W = max(3, args.steps // 4), max(args.warmup, 6)
    out = {"unit": UNIT}
    for name, cp in (("cd4", 0), ("compact6", 1)):
        case = I.tgv_case(128, 4, "CAA", viscous=False, compact=cp)
        case = case.replace(dt=I.cfl_dt(case, I.tgv_state(case), 0.25))
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            s = cfs.Solver(case, graph=True, stream=st)
            try:
                s.set_schedule()
                s.set_state(I.tgv_state(case))
                s.step(W)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(st)
                s.step(K)
                e1.record(st)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / K
                cfs.cfs_set_timing(s.ctx, True)
                s.step(2)
                kt = cfs.cfs_get_timing(s.ctx)
                cfs.cfs_set_timing(s.ctx, False)
                fin = bool(np.all(np.isfinite(s.get_state())))
            finally:
                s.close()
        out[name] = {"value": case.npts * case.stages / (ms * 1e-3) / 1e6, "ms_per_step": ms, "finite": fin,
                     "per_kernel_ms_per_step": {k: round(v[0] / 2, 4) for k, v in kt.items() if v[1]}}
    out["compact_over_cd4_time"] = out["compact6"]["ms_per_step"] / out["cd4"]["ms_per_step"]
    out["workload"] = ("Euler TGV 128^3, 4^3 sub-domains of 32^3, CAA-AT L=4 at CFL 0.25, filter; sixth-order compact "
                       "(Eq. 2, alpha 1/3, halo depth 4) against CD4; per-kernel: stage_update = compact line solves + "
                       "update")
    return out


def static_diagnostics_form():
    """Latency of the allocation-free diagnostics (cfs_diagnostics_static) at its size limit: a
    256^3 TGV state (16.8 M points, the 4 MiB scratch full), CUDA events around each call, median
    of 10 after 2 warm-up calls, beside cfs_diagnostics of a context on the same state."""
    import torch
    from paper_2506_03027_gb300 import cfs
    from paper_2506_03027_gb300 import inputs as I
    c = I.tgv_case(256, 8, "SA")
    U = torch.from_numpy(I.tgv_state(c)).cuda()
    out = torch.empty(8, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    ts = []
    for it in range(12):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        cfs.cfs_diagnostics_static(U.data_ptr(), c.nx, c.ny, c.nz, (c.dx, c.dy, c.dz), 4, out.data_ptr(), st.cuda_stream)
        e1.record(st)
        torch.cuda.synchronize()
        if it >= 2:
            ts.append(e0.elapsed_time(e1))
    return {"ms_median": statistics.median(ts), "ms_min": min(ts), "points": c.npts,
            "workload": "TGV 256^3 state (the size limit), order 4; CUDA events around each call"}


def oracle_sample(case, nsteps):
    """Time `nsteps` asynchronous oracle steps of the workload (starting after the warm-up with a
    history of copies of the initial state: the cost does not depend on the values)."""
    from oracle import oracle as orc
    from paper_2506_03027_gb300 import inputs as I
    U0 = I.tgv_state(case)
    R = 3 + case.levels + 1
    hist = np.broadcast_to(U0, (R,) + U0.shape).copy()
    n0 = case.levels
    delays = I.saa_delays(case, n0 + nsteps)
    t0 = time.perf_counter()
    orc.run(case, U0, nsteps, delays=delays, n0=n0, hist=hist)
    return time.perf_counter() - t0


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the baseline record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu model")):
                    return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def cpu_baseline(case):
    """The oracle on the host cores: one asynchronous step of the full workload with OpenMP over
    the sub-domains on every core, and one on a single thread."""
    from oracle import oracle as orc
    orc.build()
    steps = 1
    cores = orc.num_threads()
    dt = oracle_sample(case, steps)
    orc.set_num_threads(1)
    try:
        dt1 = oracle_sample(case, steps)
    finally:
        orc.set_num_threads(cores)
    return {"value": case.npts * case.stages * steps / dt / 1e6, "unit": UNIT, "cores": cores,
            "kind": "oracle", "cpu_model": cpu_model(),
            "single_thread": {"value": case.npts * case.stages * steps / dt1 / 1e6, "cores": 1, "seconds": dt1},
            "sample": f"{steps} asynchronous step(s) of the full 128^3 workload (SAA-AT, filter): {dt:.1f} s on "
                      f"{cores} threads, {dt1:.1f} s on one"}


def run_reference(args):
    from oracle import oracle as orc
    orc.build()
    case = workload(args.schedule)
    for _ in range(args.warmup):
        oracle_sample(case, 1)
    ts = [oracle_sample(case, 1) for _ in range(args.steps)]
    tot = sum(ts)
    value = case.npts * case.stages * args.steps / tot / 1e6
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "Taylor-Green vortex NS 128^3, 4x4x4 sub-domains of 32^3, SAA-AT delays 0..3, "
                                   "LSERK4-CD4-AT4, 10th-order filter alpha_f 0.499",
                       "grid": [case.nx, case.ny, case.nz], "subdomains": case.nsub, "schedule": args.schedule},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": orc.num_threads(), "kind": "oracle",
                             "sample": f"{args.steps} full asynchronous steps of the 128^3 workload"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=6)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--schedule", default="SAA", choices=["SA", "CAA", "SAA"])
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-halo form (trains a network)")
    ap.add_argument("--grid", type=int, default=128, help="grid points per axis (profiling runs only)")
    ap.add_argument("--split", type=int, default=4, help="sub-domains per axis (profiling runs only)")
    ap.add_argument("--tiles", default="", help="fy,zc,threads launch shapes of the main path (profiling runs only)")
    ap.add_argument("--only-form", default="", choices=["", "cgrid_naca0012", "cgrid_naca0012_fp32_intermediates",
                                                        "learned_halo", "compact_euler", "batched_blocks_curvilinear",
                                                        "static_diagnostics", "fp32_intermediates_256"],
                    help="run one form alone and print its result (profiling runs only; --tiles skips its autotuning)")
    ap.add_argument("--cgrid-half", action="store_true",
                    help="with --only-form: the C-grid at half the points per direction (profiling runs only)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.only_form:
        import torch
        torch.cuda.init()
        from paper_2506_03027_gb300 import build as B
        B.build()
        if args.only_form == "learned_halo":
            print(json.dumps(learned_form(args)), flush=True)
            return
        if args.only_form == "compact_euler":
            print(json.dumps(compact_form(args)), flush=True)
            return
        if args.only_form == "batched_blocks_curvilinear":
            print(json.dumps(batched_form(args, 0, curvilinear=True)), flush=True)
            return
        if args.only_form == "static_diagnostics":
            print(json.dumps(static_diagnostics_form()), flush=True)
            return
        if args.only_form == "fp32_intermediates_256":
            print(json.dumps(precision_form_256(args)), flush=True)
            return
        print(json.dumps(cgrid_form(args, 1 if args.only_form.endswith("fp32_intermediates") else 0)), flush=True)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    line = run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
