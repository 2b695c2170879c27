#!/usr/bin/env python3
"""Benchmark of the GB300 Teukolsky Lax-Wendroff solver.

One benchmark step is one whole solve of the workload through the C ABI:
Kerr coefficient precompute, initial data, every outer time step with its
waveform samples, and the waveform read-out.  The default workload is the Kerr
a = 0.9 M evolution on a 25601 x 64 grid for 38400 steps (t = 600 M).

Printed: one JSON line with grid-point updates/s (value: inputs already in
HBM; e2e: host buffers, copies inside the timed region), the roofline of the
step kernel measured live with CUDA events, the clocks seen during the timed
region, and the CPU oracle timed on a bounded sample on the host cores.

``--impl reference`` times the CPU oracle instead (each step a bounded sample
of the same workload) and prints the same line with ``"impl": "reference"``.

Multi-GPU (torchrun): one solve is not split across GPUs; each rank runs
its own replica of the workload and ``value`` counts the updates of all ranks
over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from inputs import (ADJOINT_16001x128, KERR_25601x64, SCHWARZSCHILD_1601x32,  # noqa: E402
                    adjoint_target_params, batched_instances, initial_planes)

WORKLOADS = {"kerr": KERR_25601x64, "schwarzschild": SCHWARZSCHILD_1601x32,
             "batched": None, "adjoint": ADJOINT_16001x128}

# FP64 work of the step kernel per grid-point update, counted from its source:
# half node (Eq. lw1) 4 adds + 2 multiplies + 20 FMAs, node (Eq. lw2) 4 adds +
# 24 FMAs; an FMA counts 2 flops.  The adds and multiplies are issued as FMAs
# with 1 and -0 (54 DFMA instructions), so at most 98 of the 108 flops a full
# pipe would do are useful.
FP64_FLOP_PER_UPDATE = (4 + 2 + 2 * 20) + (4 + 2 * 24)          # = 98
FP64_INSTR_PER_UPDATE = 26 + 28
# adjoint step per update: 46 FMAs + 6 multiplies + 10 adds (transposed blocks
# and transposed theta couplings at the node and the half node)
ADJ_FLOP_PER_UPDATE = 2 * 46 + 6 + 10                            # = 108
ADJ_INSTR_PER_UPDATE = 62
STATE_BYTES_PER_UPDATE = {0: 64, 1: 32}                         # read u^n, write u^{n+1}
TABLE_BYTES_PER_UPDATE = {0: 21 * 8, 1: 21 * 4}                 # 11 + 10 table entries
# the four-step FP32 sweep reads the compact FP32 tables: 16 of the 21 entries
# per point (the other five are derived in the kernel)
FP32_SWEEP_TABLE_BYTES = 16 * 4
NUM_SMS = 152
FP64_FMA_PER_CLK_PER_SM = 2        # measured: 1.19 TFLOP/s at 1995 MHz on 152 SMs
FP32_FMA_PER_CLK_PER_SM = 128


# DRAM bytes per unit of work of the step kernel (one inner step of the FP64
# persistent launch, one sweep of the FP32 one: dram__bytes_read.sum +
# dram__bytes_write.sum from one ncu capture of the current kernel source),
# keyed by (workload name, precision); the capture's command and figures are in the
# named summary under profiles/.
MEASURED_TRAFFIC = {
    # one persistent launch of 200 steps: 65.775047 + 10.831660 GB, per step
    ("kerr_a0.9_25601x64_38400steps", 0): ((65.775047e9 + 10.831660e9) / 200,
                                           "profiles/lw_persistent_f64_kerr_25601x64.md"),
    # one launch of 50 sweeps of four steps: 6.726055 + 1.280336 GB
    ("kerr_a0.9_25601x64_38400steps", 1): ((6.726055e9 + 1.280336e9) / 50,
                                           "profiles/lw_multi_persistent_f32_kerr_25601x64.md"),
}
# FP32 on the Kerr workload: every inner step of the solve in one cooperative
# launch, four Lax-Wendroff steps per sweep over the grid (25601 columns: at
# least 4 per warp of 8 warps on each of the 152 SMs).
FP32_STEPS_PER_SWEEP = 4
L2_FLUSH_BYTES = 256 << 20          # twice the 129 MB L2


def _hbm_peak():
    """Measured HBM copy bandwidth of the GB300s (GB/s) and its source."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    except (OSError, ValueError, KeyError):
        return 6800.0, "6.8 TB/s (of fallback: no MEASURED_PEAKS.json)"


HBM_GBS, HBM_SRC = _hbm_peak()


class L2Flush:
    """Writes a buffer twice the size of L2 on the stream, evicting every line
    the previous step left behind."""

    def __init__(self, torch):
        self.buf = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def __call__(self):
        self.buf.zero_()


L2_NOTE = "L2 flushed (256 MB write) before every timed step, inside the timed region"


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples every 200 ms."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", self.gpu_id], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                smax.append(float(p[1]))
                power.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "power_w_max": max(power), "samples": len(sm), "reasons": sorted(reasons)}


def _gpu_id(torch, dev: int) -> str:
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(dev)


def cpu_baseline(w, sample_steps: int) -> dict:
    """The CPU oracle, as it stands, on a bounded sample of the workload."""
    import oracle
    oracle.build()
    threads = oracle.get_threads()
    sol = oracle.Solver(M=w.M, a=w.a, s=w.s, m=w.m, rs_min=w.rs_min, rs_max=w.rs_max, Nr=w.Nr,
                        Ntheta=w.Ntheta, dt=w.dt, substeps=w.substeps, variable=w.variable)
    for r, t in w.observers:
        sol.add_observer(r, t)
    re, im = initial_planes(w)
    sol.set_initial(re, im)
    t0 = time.perf_counter()
    sol.run(sample_steps)
    dt = time.perf_counter() - t0
    ups = w.points * sample_steps * w.substeps / dt
    return {"value": ups, "unit": "updates/s", "cores": threads, "kind": "oracle",
            "sample": f"first {sample_steps} of {w.steps} outer steps of {w.name} "
                      f"(time stepping only, {threads} OpenMP threads, {os.cpu_count()} host cores)",
            "seconds": dt}


def run_reference(args, w):
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    sample = args.ref_sample_steps
    import oracle
    oracle.build()
    threads = oracle.get_threads()
    sol = oracle.Solver(M=w.M, a=w.a, s=w.s, m=w.m, rs_min=w.rs_min, rs_max=w.rs_max, Nr=w.Nr,
                        Ntheta=w.Ntheta, dt=w.dt, substeps=w.substeps, variable=w.variable)
    for r, t in w.observers:
        sol.add_observer(r, t)
    re, im = initial_planes(w)
    sol.set_initial(re, im)
    for _ in range(args.warmup):
        sol.run(sample)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sol.run(sample)
    dt = time.perf_counter() - t0
    ups = w.points * sample * w.substeps * args.steps / dt
    line = {
        "impl": "reference", "metric": "grid-point updates/s", "value": ups, "unit": "updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(w, args, world),
        "cpu_baseline": {"value": ups, "unit": "updates/s", "cores": threads, "kind": "oracle",
                         "sample": f"each step: {sample} outer steps of {w.name} on the CPU oracle "
                                   f"({threads} OpenMP threads, {os.cpu_count()} host cores)"},
        "e2e": {"value": ups, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def _variant_name(w, base) -> str:
    parts = [base.name]
    if w.variable != base.variable:
        parts.append("literal" if w.variable == 0 else "regularised")
    if w.s != base.s:
        parts.append(f"s{w.s}")
    if w.substeps != base.substeps:
        parts.append(f"k{w.substeps}" if w.substeps else "kauto")
    return "_".join(parts)


def _config(w, args, world, precision=None):
    precision = args.precision if precision is None else precision
    return {"workload": w.name, "a": w.a, "M": w.M, "s": w.s, "m": w.m, "Nr": w.Nr,
            "Ntheta": w.Ntheta, "rstar": [w.rs_min, w.rs_max], "dt": w.dt,
            "outer_steps": args.outer_steps or w.steps, "substeps": w.substeps,
            "variable": "regularised" if w.variable else "literal",
            "precision": "f32" if precision else "f64",
            "observers": [list(o) for o in w.observers],
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "l2": L2_NOTE + "; working set: state 2x{:.1f} MB + tables {:.1f} MB".format(
                w.points * STATE_BYTES_PER_UPDATE[precision] / 1e6,
                w.points * TABLE_BYTES_PER_UPDATE[precision] / 1e6)}


def _clock_checked(clk):
    bad = [r for r in clk.get("reasons", []) if r in ("hw_slowdown", "hw_thermal_slowdown",
                                                      "sw_thermal_slowdown")]
    return bad


def run_batched(args, tk, torch, rank, world, local, steps=None, warmup=None, emit=True):
    """The 24-instance batch: instances sharded across ranks by cost, each
    rank's share advanced by one tk_batch (one launch per inner tick, graph
    replay, autotuned segment length); compared with running the same
    instances one after another through tk_step.  Prints the JSON line (emit)
    or returns its fields."""
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    from paper_1010_3816_gb300 import distributed as D
    inst_all = batched_instances()
    if args.instances:
        inst_all = inst_all[:args.instances]
    n_outer = args.outer_steps or 500
    mine = D.shard([w.points * w.substeps for w in inst_all], rank, world)
    inst = [inst_all[k] for k in mine]
    stream = torch.cuda.current_stream()
    solvers, planes, outs = [], [], []
    for w in inst:
        g = tk.Solver(rstar_min=w.rs_min, rstar_max=w.rs_max, Nr=w.Nr, Ntheta=w.Ntheta, dt=w.dt,
                      substeps=w.substeps, variable=w.variable, stream=stream.cuda_stream)
        g.precompute(w.a, w.M, w.s, w.m)
        re, im = initial_planes(w)
        d = (torch.from_numpy(re).cuda(), torch.from_numpy(im).cuda())
        g.set_initial(*d)
        ids = [g.add_observer(r, t) for r, t in w.observers]
        outs.append([(k, torch.empty(n_outer, dtype=torch.float64, device="cuda"),
                      torch.empty(n_outer, dtype=torch.float64, device="cuda")) for k in ids])
        solvers.append(g)
        planes.append(d)
    batch = tk.Batch(solvers)
    seg, tuned_ms = batch.tune(3)
    info = batch.info()
    updates = sum(w.points * w.substeps for w in inst) * n_outer
    ev = []

    def solve(record, batched=True):
        for g, w, d in zip(solvers, inst, planes):
            tk.tk_precompute_coeffs(g.h, w.a, w.M, w.s, w.m)
            tk.tk_set_initial_data(g.h, *d)
        if record:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        if batched:
            batch.step(n_outer)
        else:
            for g in solvers:
                g.step(n_outer)
        if record:
            e1.record(stream)
            ev.append((e0, e1))
        for g, o in zip(solvers, outs):
            for k, a, b in o:
                tk.tk_extract(g.h, k, a, b)

    flush = L2Flush(torch)
    for _ in range(warmup):
        flush()
        solve(False)
    torch.cuda.synchronize()
    D.barrier()
    clocks = ClockSampler(_gpu_id(torch, local))
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        flush()
        solve(True)
    t1.record(stream)
    torch.cuda.synchronize()
    D.barrier()
    clk = clocks.stop()
    ms = D.reduce_max(t0.elapsed_time(t1), device="cuda")
    total_updates = D.reduce_sum(updates, device="cuda")
    value = total_updates * steps / (ms * 1e-3)
    kern_s = statistics.mean(a.elapsed_time(b) for a, b in ev) * 1e-3
    # the same instances through tk_step, one after another
    solve(False, batched=False)
    torch.cuda.synchronize()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    solve(True, batched=False)
    p1.record(stream)
    torch.cuda.synchronize()
    plain = updates / (p0.elapsed_time(p1) * 1e-3)
    f_clk = (clk.get("sm_mhz") or 2070.0) * 1e6
    achieved = FP64_FLOP_PER_UPDATE * updates / kern_s / 1e12
    peak = NUM_SMS * FP64_FMA_PER_CLK_PER_SM * 2 * f_clk / 1e12
    line = None
    if rank == 0:
        line = {
            "metric": "grid-point updates/s", "value": value, "unit": "updates/s", "n_gpus": world,
            "steps": steps, "warmup": warmup, "ms_per_step": ms / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"batched_{len(inst_all)}_instances", "instances": len(inst_all),
                       "instances_on_rank0": len(inst), "outer_steps": n_outer,
                       "outer_steps_of_full_run": inst_all[0].steps,
                       "substeps_by_Ntheta": {"32": 2, "64": 4, "128": 8}, "ticks_per_outer_step": info["kmax"],
                       "segment_autotuned": seg, "tuned_ms_per_outer_step": tuned_ms,
                       "grid_blocks": info["blocks"],
                       "strategy": ("members one after another, each as one persistent launch (the tuner's "
                                    "choice: faster than the work queue here)") if seg == 0
                                   else "work queue of (member, column range) items, one launch per tick",
                       "parallelism": f"instances sharded over {world} GPUs" if world > 1 else "single GPU",
                       "l2": L2_NOTE},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "lw_persistent_kernel<double>" if seg == 0 else "batch_step_kernel<double>",
                         "peak_source": "152 SMs x 2 DFMA/clk (measured) x 2 flop x median SM clock"},
            "plain_tk_step": {"value": plain, "unit": "updates/s",
                              "what": "the same instances through tk_step one after another"},
            "ratio_vs_sequential_tk_step": (updates / kern_s) / plain,
            "cpu_baseline": None, "e2e": None, "clocks": clk,
            # per timed step: the ticks (or one persistent launch per member),
            # and per member the precompute's three launches and one read-out
            # per observer
            "gpu_launches": steps * ((len(inst) if seg == 0 else n_outer * info["kmax"]) + 3 * len(inst) +
                                     sum(len(o) for o in outs)),
        }
        if emit:
            print(json.dumps(line))
    batch.close()
    return 0 if emit else line


def run_adjoint(args, tk, torch, rank, world, local):
    """Gradient of the waveform misfit sum_t |W(t) - W_target(t)|^2 with
    respect to the amplitude, centre and width of the initial pulse: forward
    solve, then the adjoint sweep (tk_adjoint) through torch.autograd."""
    w = ADJOINT_16001x128
    # t = 400 M by default: the pulse launched at r* = 50 has passed the observer
    # at r* = 400, so the misfit and its gradient are not zero
    n_outer = args.outer_steps or 12800
    stream = torch.cuda.current_stream()
    g = tk.Solver(rstar_min=w.rs_min, rstar_max=w.rs_max, Nr=w.Nr, Ntheta=w.Ntheta, dt=w.dt,
                  substeps=w.substeps, variable=w.variable, stream=stream.cuda_stream)
    g.precompute(w.a, w.M, w.s, w.m)
    g.set_initial(*(torch.zeros((w.Ntheta, w.Nr), dtype=torch.float64, device="cuda") for _ in range(2)))
    for r, t in w.observers:
        g.add_observer(r, t)
    rs = torch.tensor(w.rs_min + np.arange(w.Nr) * w.drs, dtype=torch.float64, device="cuda")
    th = torch.tensor((np.arange(w.Ntheta) + 0.5) * (math.pi / w.Ntheta), dtype=torch.float64,
                      device="cuda")
    ang = (torch.sin(th) ** 2)[:, None]

    def planes(A, c, s):
        G = A * torch.exp(-((rs - c) ** 2) / (2.0 * s ** 2))
        re = ang * G[None, :]
        return re, torch.zeros_like(re)

    with torch.no_grad():
        tA, tc, tw = (torch.tensor(v, dtype=torch.float64, device="cuda") for v in adjoint_target_params())
        target = tk.waveforms(g, *planes(tA, tc, tw), n_outer).clone()
    ev_f, ev_b = [], []

    def gradient(record):
        p = [torch.tensor(v, dtype=torch.float64, device="cuda", requires_grad=True)
             for v in (w.amp, w.center, w.width)]
        if record:
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
        W = tk.waveforms(g, *planes(*p), n_outer)
        L = ((W - target) ** 2).sum()
        if record:
            e[1].record(stream)
        L.backward()
        if record:
            e[2].record(stream)
            ev_f.append((e[0], e[1]))
            ev_b.append((e[1], e[2]))
        return [x.grad for x in p]

    flush = L2Flush(torch)
    for _ in range(args.warmup):
        flush()
        gradient(False)
    torch.cuda.synchronize()
    clocks = ClockSampler(_gpu_id(torch, local))
    clocks.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        flush()
        grads = gradient(True)
    t1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = t0.elapsed_time(t1)
    inner = w.points * w.substeps * n_outer
    value = 2 * inner * args.steps / (ms * 1e-3)
    fwd = statistics.mean(a.elapsed_time(b) for a, b in ev_f) * 1e-3
    bwd = statistics.mean(a.elapsed_time(b) for a, b in ev_b) * 1e-3
    f_clk = (clk.get("sm_mhz") or 2070.0) * 1e6
    peak = NUM_SMS * FP64_FMA_PER_CLK_PER_SM * 2 * f_clk / 1e12
    n_inner = n_outer * w.substeps
    fwd_persistent = tk.tk_get_steps_per_launch(g.h) == -1

    def fp64_roof(kernel, flop, instr, seconds):
        launch_s = seconds / n_inner
        ach = flop * w.points / launch_s / 1e12
        return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": None, "kernel": kernel, "flop_per_update": flop,
                "fp64_issue_frac": instr * w.points / launch_s /
                (NUM_SMS * FP64_FMA_PER_CLK_PER_SM * f_clk),
                "launch_us": launch_s * 1e6,
                "peak_source": "152 SMs x 2 DFMA/clk (measured) x 2 flop x median SM clock "
                               f"{f_clk / 1e6:.0f} MHz"}
    pgrad = None
    if args.param_gradient:
        # dL/da and dL/dM of the same loss at the workload's parameters
        with torch.no_grad():
            W = tk.waveforms(g, *planes(*(torch.tensor(v, dtype=torch.float64, device="cuda")
                                          for v in (w.amp, w.center, w.width))), n_outer)
            dW = (2.0 * (W - target)).cpu().numpy()           # [obs][samples][2]
        pgrad = {"checkpoint_every_outer_steps": args.checkpoint_every}
        for name in ("a", "M"):
            torch.cuda.synchronize()
            t0p = time.perf_counter()
            pgrad["dL_d" + name] = g.param_gradient(name, dW, args.checkpoint_every)
            pgrad["seconds_" + name] = time.perf_counter() - t0p
    if rank == 0:
        line = {
            "metric": "grid-point updates/s (forward + adjoint)", "value": value, "unit": "updates/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": w.name, "Nr": w.Nr, "Ntheta": w.Ntheta, "a": w.a,
                       "outer_steps": n_outer, "outer_steps_of_full_run": w.steps,
                       "substeps": w.substeps, "loss": "sum_t |W(t) - W_target(t)|^2 at (400, pi/2)",
                       "gradient_wrt": ["amplitude", "centre", "width", "initial planes"],
                       "parallelism": "single GPU", "l2": L2_NOTE},
            "forward_updates_per_s": inner / fwd, "adjoint_updates_per_s": inner / bwd,
            "roofline_adjoint": fp64_roof("lw_adjoint_persistent_kernel<double>" if fwd_persistent
                                          else "lw_adjoint_kernel<double>", ADJ_FLOP_PER_UPDATE,
                                          ADJ_INSTR_PER_UPDATE, bwd),
            "grad": [float(x) for x in grads], "param_gradient": pgrad,
            "roofline": fp64_roof("lw_persistent_kernel<double>" if fwd_persistent else "lw_step_kernel<double>",
                                  FP64_FLOP_PER_UPDATE, FP64_INSTR_PER_UPDATE, fwd),
            "cpu_baseline": None, "e2e": None, "clocks": clk,
            # per timed step: the forward solve and the adjoint sweep, each one
            # persistent launch, or one launch per inner step
            "gpu_launches": args.steps * (2 if fwd_persistent else 2 * n_inner),
        }
        print(json.dumps(line))
    g.close()
    return 0


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3,
                    help=">= 3 for a valid measurement (fewer only for profiling runs)")
    ap.add_argument("--impl", default="tk", choices=["tk", "reference"])
    ap.add_argument("--workload", default="kerr", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1])
    ap.add_argument("--outer-steps", type=int, default=0,
                    help="outer steps per solve (default: the workload's); for profiling runs")
    ap.add_argument("--cpu-sample-steps", type=int, default=150)
    ap.add_argument("--ref-sample-steps", type=int, default=40)
    ap.add_argument("--variable", choices=["regularised", "literal"], default=None,
                    help="angular variable (default: the workload's); the literal variable "
                         "needs more substeps, see --substeps")
    ap.add_argument("--spin-weight", type=int, default=None,
                    help="spin weight s (default: the workload's -2; 0 is the scalar field)")
    ap.add_argument("--substeps", type=int, default=None,
                    help="Lax-Wendroff steps per outer step (default: the workload's; 0: from "
                         "the stability bound)")
    ap.add_argument("--param-gradient", action="store_true",
                    help="adjoint workload: also dL/da and dL/dM through checkpointed "
                         "recomputation (after the timed region)")
    ap.add_argument("--checkpoint-every", type=int, default=150,
                    help="outer steps between checkpoints for --param-gradient")
    ap.add_argument("--instances", type=int, default=0,
                    help="batched workload: the first N of its 24 instances (profiling runs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra-arms", action="store_true",
                    help="Kerr FP64 run: skip the FP32 and batched arms that follow it")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    if w is not None:
        if args.variable is not None:
            w = w.with_(variable=1 if args.variable == "regularised" else 0)
        if args.spin_weight is not None:
            w = w.with_(s=args.spin_weight)
        if args.substeps is not None:
            w = w.with_(substeps=args.substeps)
        if w != WORKLOADS[args.workload]:
            w = w.with_(name=_variant_name(w, WORKLOADS[args.workload]))
    if args.impl == "reference":
        w = w or batched_instances()[2]
        if w.substeps == 0:
            raise SystemExit("the oracle takes an explicit number of substeps (--substeps k)")
        return run_reference(args, w)

    import torch
    import paper_1010_3816_gb300 as tk

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    tk.load_library()
    if args.workload in ("batched", "adjoint"):
        fn = run_batched if args.workload == "batched" else run_adjoint
        rc = fn(args, tk, torch, rank, world, local)
        if dist:
            dist.destroy_process_group()
        return rc
    main_arm = measure_solve(args, tk, torch, w, args.precision, args.steps, args.warmup, rank,
                             world, local, dist, not args.no_e2e)
    line = None
    if rank == 0:
        cpu = None if args.no_cpu_baseline or world > 1 else cpu_baseline(main_arm["w"],
                                                                           args.cpu_sample_steps)
        line = {
            "metric": "grid-point updates/s", "value": main_arm["value"], "unit": "updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": main_arm["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision else "f64", "data": "synthetic",
            "config": _config(main_arm["w"], args, world, args.precision),
            "roofline": main_arm["roofline"], "roofline_hbm": main_arm["roofline_hbm"],
            "parity_vs_oracle_full_run": main_arm["parity"],
            "cpu_baseline": cpu, "e2e": main_arm["e2e"], "clocks": main_arm["clocks"],
            "gpu_launches": main_arm["gpu_launches"],
        }
    # the metric's other two forms on the same GPU, after the FP64 arm: FP32 at
    # its stated waveform error, and the batched instances against the same
    # instances through tk_step one after another
    extra = (args.workload == "kerr" and args.precision == 0 and not args.no_extra_arms and
             w == WORKLOADS["kerr"] and not args.outer_steps)
    if extra:
        f32 = measure_solve(args, tk, torch, w, 1, args.steps, args.warmup, rank, world, local, dist,
                            not args.no_e2e)
        if rank == 0:
            line["fp32"] = {
                "value": f32["value"], "unit": "updates/s", "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": f32["ms_per_step"],
                "ratio_vs_fp64": f32["value"] / main_arm["value"],
                "e2e": f32["e2e"],
                "e2e_ratio_vs_fp64": (f32["e2e"]["value"] / main_arm["e2e"]["value"]
                                      if f32["e2e"] and main_arm["e2e"] else None),
                "error_vs_fp64_oracle_full_run": f32["parity"],
                "roofline": f32["roofline"], "roofline_hbm": f32["roofline_hbm"],
                "clocks": f32["clocks"], "gpu_launches": f32["gpu_launches"],
                "config": _config(w, args, world, 1)}
        bsteps = min(args.steps, 5)
        bat = run_batched(args, tk, torch, rank, world, local, steps=bsteps, warmup=3, emit=False)
        if rank == 0:
            line["batched"] = bat
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


# Stored full-length oracle run of the Kerr workload (tests/golden/make_kerr_golden.py).
GOLDEN_KERR = os.path.join(ROOT, "tests", "golden", "kerr_25601x64_oracle.npz")


def _parity_full_run(w, waves):
    """Relative L2 of the waveforms against the oracle's stored full run of the
    Kerr workload, or None when this solve is not that run."""
    if w != WORKLOADS["kerr"] or not os.path.exists(GOLDEN_KERR):
        return None
    ref = np.load(GOLDEN_KERR)
    out = {"reference": "tests/golden/kerr_25601x64_oracle.npz (FP64 CPU oracle, all 38400 outer "
                        "steps)"}
    for k, key in enumerate(("wave0", "wave1")):
        out[key + "_rel_l2"] = float(np.linalg.norm(waves[k] - ref[key]) / np.linalg.norm(ref[key]))
    out["observers"] = [list(o) for o in w.observers]
    return out


def measure_solve(args, tk, torch, w, precision, steps, warmup, rank, world, local, dist, do_e2e):
    """Whole solves of workload w at the given precision: `warmup` untimed,
    then `steps` timed (device-resident inputs, L2 flushed before each), then
    the same through host buffers (e2e).  Returns the numbers of one arm."""
    n_outer = args.outer_steps or w.steps
    stream = torch.cuda.current_stream()
    solver = tk.Solver(rstar_min=w.rs_min, rstar_max=w.rs_max, Nr=w.Nr, Ntheta=w.Ntheta, dt=w.dt,
                       substeps=w.substeps, variable=w.variable, precision=precision,
                       stream=stream.cuda_stream)
    if w.substeps == 0:
        # substeps chosen by the solver's stability bound at the precompute
        solver.precompute(w.a, w.M, w.s, w.m)
        w = w.with_(substeps=solver.substeps)
    updates = w.points * n_outer * w.substeps
    # the library's default: FP32 runs the solve's inner steps as sweeps of
    # four in one persistent launch (whole outer steps), the rest as pairs in
    # a second one and an odd last step alone; FP64 runs them all in one
    # persistent launch (read back from the library)
    spl = FP32_STEPS_PER_SWEEP if precision == 1 else 1
    inner_steps = n_outer * w.substeps
    # FP64: every step of the solve in one persistent launch, unless the
    # library chose one launch per step for this grid (read back)
    fp64_persistent = precision == 0 and tk.tk_get_steps_per_launch(solver.h) == -1
    if precision == 1:
        unit = w.substeps // math.gcd(spl, w.substeps)
        sweeps = inner_steps // spl // unit * unit
        rest = inner_steps - sweeps * spl
        step_launches = int(sweeps > 0) + int(rest >= 2) + rest % 2
    elif fp64_persistent:
        step_launches = 1
    else:
        step_launches = inner_steps
    launches_per_solve = 3 + step_launches + len(w.observers)
    re, im = initial_planes(w)
    d_re = torch.from_numpy(re).cuda()
    d_im = torch.from_numpy(im).cuda()
    obs_out = [(torch.empty(n_outer, dtype=torch.float64, device="cuda"),
                torch.empty(n_outer, dtype=torch.float64, device="cuda")) for _ in w.observers]
    solver.precompute(w.a, w.M, w.s, w.m)
    solver.set_initial(d_re, d_im)
    obs_ids = [solver.add_observer(r, t) for r, t in w.observers]

    ev_step = []

    def solve_device(record: bool):
        tk.tk_precompute_coeffs(solver.h, w.a, w.M, w.s, w.m)
        tk.tk_set_initial_data(solver.h, d_re, d_im)
        if record:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        tk.tk_step(solver.h, n_outer)
        if record:
            e1.record(stream)
            ev_step.append((e0, e1))
        for k, (a, b) in zip(obs_ids, obs_out):
            tk.tk_extract(solver.h, k, a, b)

    flush = L2Flush(torch)
    for _ in range(warmup):
        flush()
        solve_device(False)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(_gpu_id(torch, local))
    clocks.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(steps):
        flush()
        solve_device(True)
    t_end.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = t_start.elapsed_time(t_end)
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * updates * steps / (ms * 1e-3)
    step_ms = [a.elapsed_time(b) for a, b in ev_step]
    kern_s = statistics.mean(step_ms) * 1e-3 / (n_outer * w.substeps)   # per inner step
    pts = w.points
    f_clk = (clk.get("sm_mhz") or 2070.0) * 1e6
    traffic, traffic_src = MEASURED_TRAFFIC.get((w.name, precision), (None, None))
    if precision == 0:
        achieved = FP64_FLOP_PER_UPDATE * pts / kern_s / 1e12
        peak = NUM_SMS * FP64_FMA_PER_CLK_PER_SM * 2 * f_clk / 1e12
        probe = fp64_probe(tk, f_clk)
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": "lw_persistent_kernel<double>" if fp64_persistent else "lw_step_kernel<double>",
                "peak_source": "152 SMs x 2 DFMA/clk x 2 flop x median SM clock "
                               f"{f_clk / 1e6:.0f} MHz (GB300 FP64 FMA issue rate; "
                               "profiles/fp64_pipe_peak.md)",
                "peak_measured": probe["tflops"],
                "frac_of_measured": achieved / probe["tflops"],
                "peak_measured_source": "tk_probe_fp64_fma in this run: " + probe["how"],
                "traffic_source": traffic_src, "flop_per_update": FP64_FLOP_PER_UPDATE,
                "fp64_issue_frac": FP64_INSTR_PER_UPDATE * pts / kern_s /
                (NUM_SMS * FP64_FMA_PER_CLK_PER_SM * f_clk),
                "step_us": kern_s * 1e6,
                "launch_us": kern_s * 1e6 * (inner_steps if fp64_persistent else 1)}
    else:
        # the unit of work is one sweep of FP32_STEPS_PER_SWEEP inner steps: it
        # reads u^n and the compact tables once and writes u^{n+4}; algorithmic
        # bytes per sweep = (32 + 64) B per point.  All sweeps of the solve run
        # in one launch.
        sweep_s = spl * kern_s
        alg = (STATE_BYTES_PER_UPDATE[1] + FP32_SWEEP_TABLE_BYTES) * pts
        achieved = alg / sweep_s / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": HBM_GBS, "unit": "GB/s",
                "frac": achieved / HBM_GBS, "traffic": traffic,
                "kernel": "lw_multi_persistent_kernel<float>",
                "algorithmic_bytes_per_sweep": alg, "inner_steps_per_sweep": spl,
                "peak_source": HBM_SRC,
                "traffic_source": traffic_src, "sweep_us": sweep_s * 1e6}
    sb = STATE_BYTES_PER_UPDATE[precision] * pts / kern_s / 1e9
    tb = TABLE_BYTES_PER_UPDATE[precision] * pts / kern_s / 1e9
    roof_hbm = {"bound": "hbm", "achieved": sb, "peak": HBM_GBS, "unit": "GB/s",
                "frac": sb / HBM_GBS, "state_bytes_per_update": STATE_BYTES_PER_UPDATE[precision],
                "table_gbs": tb, "table_bytes_per_update": TABLE_BYTES_PER_UPDATE[precision],
                "peak_source": HBM_SRC}

    # end to end through the public API: host input planes (pinned), host waveform read-back
    e2e = None
    if do_e2e:
        h_re = torch.from_numpy(re).pin_memory()
        h_im = torch.from_numpy(im).pin_memory()
        h_out = [(np.zeros(n_outer), np.zeros(n_outer)) for _ in w.observers]
        h2d = 2 * re.nbytes
        d2h = sum(2 * 8 * n_outer for _ in w.observers)

        def solve_host():
            tk.tk_precompute_coeffs(solver.h, w.a, w.M, w.s, w.m)
            tk.tk_set_initial_data(solver.h, h_re.numpy(), h_im.numpy())
            tk.tk_step(solver.h, n_outer)
            for k, (a, b) in zip(obs_ids, h_out):
                tk.tk_extract(solver.h, k, a, b)

        solve_host()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(steps):
            flush()
            solve_host()
        torch.cuda.synchronize()
        es = time.perf_counter() - t0
        if dist:
            t = torch.tensor([es], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            es = float(t.item())
        e2e = {"value": world * updates * steps / es, "unit": "updates/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": 1e3 * es / steps}

    solver.check_finite()
    parity = None
    if rank == 0 and not args.outer_steps:
        parity = _parity_full_run(w, [solver.waveform(k) for k in obs_ids])
    solver.close()
    return {"w": w, "value": value, "ms_per_step": ms / steps, "roofline": roof,
            "roofline_hbm": roof_hbm, "e2e": e2e, "clocks": clk, "parity": parity,
            "gpu_launches": launches_per_solve * steps}


def fp64_probe(tk, f_clk):
    """The FP64 FMA pipe's rate measured by the library's microbenchmark
    (one 512-thread block per SM, 8 independent FMA chains per thread)."""
    iters = 1 << 17
    s, flop = tk.tk_probe_fp64_fma(1, 512, iters)
    tf = flop / s / 1e12
    return {"tflops": tf, "dfma_per_clk_per_sm": flop / 2 / s / (NUM_SMS * f_clk),
            "how": f"{flop:.3e} flop in {s * 1e3:.1f} ms ({flop / 2 / s / (NUM_SMS * f_clk):.3f} "
                   f"DFMA/clk/SM at {f_clk / 1e6:.0f} MHz)"}

if __name__ == "__main__":
    sys.exit(main())
