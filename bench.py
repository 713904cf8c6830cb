#!/usr/bin/env python3
"""Benchmark of the fused nodal IP-DG residual + LSRK stage on GB300.

Metric: DOF-stage updates per second (one DOF = one conserved scalar at one
node; one DOF-stage = that DOF carried through one RK stage: residual
evaluation and register update).  Workload: isentropic vortex, p = 4
(Np = 15), periodic square of 128 x 128 split quads (K = 32,768), mu = 1e-3,
advanced by the five-stage 2N-storage scheme; the mixed path (FP32
arithmetic, FP64 state, pressure and registers) is the headline, the plain
FP64 path is reported beside it.  A 512 x 512 variant (K = 524,288, working
set well above L2) is reported for the roofline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one rank per GPU) every rank runs an independent
replica (the path needs no exchange between problems); the value is the
total over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF-stage updates/s at p=4, mixed vs FP64 GPU path, and % of GB300 HBM roofline"
UNIT = "DOF-stage/s"
P = 4
NP = (P + 1) * (P + 2) // 2
L2_FLUSH_BYTES = 512 << 20
# HBM traffic of one stage launch that the algorithm needs: read K0, K1 and
# write K0, K1 (FP64, 32 B per DOF; the first stage does not read K1), plus
# the FP32 geometry record (64 B) and the connectivity record (16 B) of each
# element.
GEO_BYTES_MIXED = 64 + 16
GEO_BYTES_FP64 = 128 + 16


K_BENCH = 2 * 128 * 128
CONFIG = {"workload": "isentropic vortex, p=4 (Np=15), periodic [0,10]^2, 128x128 quads "
                      "split SW-NE (K=32768), mu=1e-3, CFL 0.3, 5-stage 2N-storage RK",
          "K": K_BENCH, "p": 4, "dofs": 4 * K_BENCH * 15,
          "precision": "mixed (FP32 arithmetic; FP64 state, pressure, RK registers)",
          "l2": "flushed (512 MB write) before every timed step; the 31 MB working set "
                "stays in L2 across the 5 stages of a step"}


# FP64 peak for the FP64 path's roofline: the GB300's nominal FP64 rate
# (a DFMA microbenchmark measured 1.18-1.20 TFLOP/s on this GPU)
FP64_PEAK_GFLOPS = 1250.0


def algorithmic_flops_per_dof_stage(p):
    """Floating-point operations of one DOF-stage of the method, counted by
    phase per element and divided by its 4 Np DOFs: broken gradient (two
    Np x Np contractions per field, then the metric terms), the volume flux
    at every node (primitives, pressure, advective and viscous fluxes,
    contravariant components: about 96), the divergence (two contractions),
    the face flux at every face node of each side (Roe flux, two penalty
    norms, normal fluxes, jump: about 250), the lift (Np x 3 Nfp per field)
    and the register update (2 FMA per DOF).  At p = 4: about 246."""
    Np, NF = (p + 1) * (p + 2) // 2, 3 * (p + 1)
    grad = 2 * 4 * Np * Np * 2 + 4 * Np * 6
    vol = 96 * Np
    div = 2 * 4 * Np * Np * 2
    face = 250 * NF
    lift = 4 * Np * NF * 2
    upd = 16 * Np
    return (grad + vol + div + face + lift + upd) / (4.0 * Np)


def algorithmic_bytes_per_step(K, geo_bytes):
    dof = 4 * K * NP
    state = dof * (24 + 4 * 32)          # stage 1 skips the K1 read
    return state + 5 * K * geo_bytes


# the sources each mixed stage-kernel shape is compiled from
KERNEL_FILES = {
    1: ("dg_stage.cuh", "dg_stage_mixed.cuh", "dg_device.cuh", "stage_mixed.cu"),
    2: ("dg_stage.cuh", "dg_stage_mixed.cuh", "dg_stage_mixed2.cuh", "dg_device.cuh", "stage_mixed.cu"),
    3: ("dg_stage.cuh", "dg_stage_mixed.cuh", "dg_stage_tc.cuh", "dg_stage_tc_body.inc", "pair2.cuh", "dg_device.cuh",
        "stage_tc.cu"),
}


def code_only(text):
    """C++ source without comments and blank space (a comment edit does not
    change the kernel)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_hash(variant=2):
    h = hashlib.sha256()
    for f in KERNEL_FILES[variant]:
        with open(os.path.join(ROOT, "paper_2508_17917_gb300", "csrc", f)) as fh:
            h.update(code_only(fh.read()).encode())
    return h.hexdigest()[:16]


KERNEL_OF_VARIANT = {1: "dg::stage_mixed_kernel<4, false>", 2: "dg::stage_mixed2_kernel<4, false>",
                     3: "dg::stage_tc_kernel<4, false, false, false>"}
SHAPE_OF_VARIANT = {1: "one node per thread", 2: "two nodes per thread",
                    3: "one warp per two elements, tensor-core contractions"}


def traffic_record_path():
    return os.path.join(ROOT, "profiles", "stage_kernel_traffic.json")


def recorded_traffic(variant):
    """DRAM bytes per DOF-stage of the mixed stage kernel in use, from the
    record `--record-traffic` writes from an ncu capture, if that capture was
    taken on the current kernel source."""
    path = traffic_record_path()
    if not os.path.isfile(path) or variant not in KERNEL_FILES:
        return None
    rec = json.load(open(path)).get(str(variant))
    if not rec or rec.get("kernel_hash") != kernel_hash(variant):
        return None
    return float(rec["dram_bytes_per_dof_stage"])


_BYTE_UNITS = {"byte": 1.0, "kbyte": 1e3, "mbyte": 1e6, "gbyte": 1e9, "tbyte": 1e12}


def ncu_dram_bytes(csv_path, kernel_regex):
    """dram__bytes_read.sum + dram__bytes_write.sum of every launch whose name
    matches kernel_regex, from `ncu -i REP --page raw --csv` output."""
    import csv
    rows = list(csv.reader(open(csv_path)))
    head = next(i for i, r in enumerate(rows) if "Kernel Name" in r and "dram__bytes_read.sum" in r)
    names, units = rows[head], rows[head + 1]
    col = {n: i for i, n in enumerate(names)}
    out = []
    for r in rows[head + 2:]:
        if len(r) != len(names) or not re.search(kernel_regex, r[col["Kernel Name"]]):
            continue
        tot = 0.0
        for m in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            tot += float(r[col[m]].replace(",", "")) * _BYTE_UNITS[units[col[m]].strip().lower()]
        out.append(tot)
    return out


def record_traffic(args):
    """Write the DRAM bytes per DOF-stage of one captured stage launch of the
    mixed kernel (variant args.variant) into the traffic record, keyed by the
    kernel's source hash."""
    if args.variant not in KERNEL_FILES:
        raise SystemExit("--record-traffic needs --variant 1, 2 or 3")
    kname = KERNEL_OF_VARIANT[args.variant].split("<")[0].replace("dg::", "")
    launches = ncu_dram_bytes(args.record_traffic, kname)
    if not launches:
        raise SystemExit(f"no {kname} launch with DRAM counters in {args.record_traffic}")
    dofs = 4 * args.record_k * NP
    path = traffic_record_path()
    rec = json.load(open(path)) if os.path.isfile(path) else {}
    rec[str(args.variant)] = {
        "kernel": KERNEL_OF_VARIANT[args.variant], "kernel_hash": kernel_hash(args.variant),
        "dram_bytes_per_dof_stage": launches[0] / dofs, "launch_bytes": launches[0], "K": args.record_k,
        "note": "a stage-2..5 launch (reads K1); from " + os.path.basename(args.record_traffic)}
    json.dump(rec, open(path, "w"), indent=1, sort_keys=True)
    print(json.dumps(rec[str(args.variant)]))


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[4], parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        pmax = max(r[2] for r in rows)
        loaded = [r for r in rows if r[2] > 0.5 * pmax] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in loaded for i, v in enumerate(r[4]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": rows[0][1],
                "reasons": reasons, "samples": len(rows), "samples_under_load": len(loaded),
                "power_w_max": pmax}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def slowest_rank_ms(local_ms, device="cpu"):
    """Max over the ranks of a timed region (ms); the local value when the
    job is not distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(local_ms)
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank, ws, total_ms):
    """Whole-job throughput of ws independent replicas: the units all ranks
    processed over the slowest rank's time."""
    return ws * units_per_rank / (total_ms * 1e-3)


def vortex_problem(n):
    import dg_inputs
    return dg_inputs.periodic_square(n)


def timed_steps(dg, torch, solver, dt, steps, warmup, flush, stream):
    """Per-step CUDA-event times (ms) with an L2 flush before every step."""
    for _ in range(warmup):
        solver.step(0.0, dt)
    torch.cuda.synchronize()
    evs = []
    n0 = solver.launches
    for _ in range(steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        solver.step(0.0, dt)
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    launches = solver.launches - n0
    return [a.elapsed_time(b) for a, b in evs], launches


def run_ours(args):
    import numpy as np
    import torch

    import dg_inputs
    import paper_2508_17917_gb300 as dg
    from dg_inputs.states import to_kcn

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    mesh = vortex_problem(128)
    K = mesh.K
    dof = 4 * K * NP
    results = {}
    solvers = {}
    for prec in ("mixed", "fp64"):
        s = dg.Solver(mesh, P, prec, stream=sh, mu=1e-3)
        if prec == "mixed" and args.variant:
            # a forced tile shape (profiling runs: timing under a profiler
            # would mislead the first-step tuner)
            s.set_variant(args.variant)
        x, y = s.node_coords()
        U0 = dg_inputs.perturb(to_kcn(dg_inputs.isentropic_vortex(x, y)), seed=0)
        s.set_state(U0)
        dt = s.dt(0.3)
        solvers[prec] = (s, U0, dt)

    # --- headline: mixed path, clocks sampled during the timed region
    s, U0, dt = solvers["mixed"]
    s.set_state(U0)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        times, launches = timed_steps(dg, torch, s, dt, args.steps, args.warmup, flush, stream)
    torch.cuda.synchronize()
    total_ms = slowest_rank_ms(sum(times), device="cuda")
    if ws > 1:
        torch.distributed.barrier()
    ok = s.check_finite()
    value = replica_value(dof * 5 * args.steps, ws, total_ms)
    ms_step = total_ms / args.steps
    stage_ms = ms_step / 5.0
    peak, peak_kind = measured_peaks()
    bytes_step = algorithmic_bytes_per_step(K, GEO_BYTES_MIXED)
    achieved = bytes_step / 5.0 / (stage_ms * 1e-3) / 1e9
    variant = s.variant
    traffic = recorded_traffic(variant)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_kind": peak_kind,
                # the recorded figure is a stage-2 launch; stage 1 does not
                # read K1 (8 B per DOF less): averaged over the step's launches
                "traffic": ((traffic - 8.0 / 5.0) * dof) if traffic is not None else None,
                "algorithmic_bytes_per_launch": bytes_step / 5.0,
                "kernel": KERNEL_OF_VARIANT.get(variant, str(variant)),
                "tile_shape": SHAPE_OF_VARIANT.get(variant, str(variant))}

    # --- FP64 path, same workload
    s64, U64, dt64 = solvers["fp64"]
    s64.set_state(U64)
    t64, _ = timed_steps(dg, torch, s64, dt64, max(3, args.steps // 20), 2, flush, stream)
    v64 = dof * 5 * len(t64) / (sum(t64) * 1e-3)
    fl64 = algorithmic_flops_per_dof_stage(P)
    roof64 = {"bound": "alu", "achieved": fl64 * v64 / 1e9, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
              "frac": fl64 * v64 / 1e9 / FP64_PEAK_GFLOPS,
              "peak_kind": "nominal GB300 FP64 rate (DFMA probe: 1.18-1.20 TFLOP/s)",
              "flops_per_dof_stage": fl64, "kernel": "dg::stage_kernel<4, double>"}

    # --- the same mixed path with the viscous vortex source (config 2's source
    #     term, S = -div F_v of the advected vortex, one source kernel per stage)
    s.set_source(dg.DG_SOURCE_VORTEX, (5.0, 5.0, 5.0, 10.0, 0.3 * 1.4 ** 0.5, 0.0))
    s.set_state(U0)
    tsrc, lsrc = timed_steps(dg, torch, s, dt, max(5, args.steps // 10), 3, flush, stream)
    s.set_source(dg.DG_SOURCE_NONE)
    vsrc = dof * 5 * len(tsrc) / (sum(tsrc) * 1e-3)
    with_source = {"workload": "same, with the viscous vortex source evaluated at every stage's time",
                   "value": vsrc, "unit": UNIT, "ms_per_step": sum(tsrc) / len(tsrc),
                   "with_over_without": vsrc / (value / ws), "launches_per_step": lsrc / len(tsrc)}

    # --- over-integration (FP64 path): the volume flux on a collapsed Gauss
    #     rule of degree min(3p, 15) instead of at the nodes, same workload
    s64.set_overint(True)
    s64.set_state(U64)
    toi, _ = timed_steps(dg, torch, s64, dt64, max(3, args.steps // 100), 2, flush, stream)
    s64.set_overint(False)
    voi = dof * 5 * len(toi) / (sum(toi) * 1e-3)
    overint = {"workload": f"same mesh and state, FP64 path, volume flux integrated with a collapsed Gauss rule "
                           f"of degree {dg.dg_overint_degree(P)}",
               "value": voi, "unit": UNIT, "ms_per_step": sum(toi) / len(toi), "over_nodal": voi / v64}

    # --- fused steps: the same mixed path as one cooperative launch per step
    s.set_fused(True)
    s.set_state(U0)
    tf, lf = timed_steps(dg, torch, s, dt, max(5, args.steps // 10), 5, flush, stream)
    s.set_fused(False)
    fused = {"workload": "same mesh, state and kernel; five stages per cooperative launch with grid barriers",
             "value": dof * 5 * len(tf) / (sum(tf) * 1e-3), "unit": UNIT, "ms_per_step": sum(tf) / len(tf),
             "launches_per_step": lf / len(tf)}

    # --- the tensor-core kernel forced (the tuner keeps the faster shape)
    stc = dg.Solver(mesh, P, "mixed", stream=sh, mu=1e-3)
    stc.set_variant(3)
    stc.set_state(U0)
    ttc, _ = timed_steps(dg, torch, stc, dt, max(5, args.steps // 10), 5, flush, stream)
    vtc = dof * 5 * len(ttc) / (sum(ttc) * 1e-3)
    tc = {"workload": "same mesh, state and time step; Dr / Ds / LIFT products as mma.sync TF32 "
                      "(three products of split operands), one warp per two elements",
          "value": vtc, "unit": UNIT, "ms_per_step": sum(ttc) / len(ttc), "tc_over_tuned": vtc / (value / ws),
          "kernel": KERNEL_OF_VARIANT[3], "tuned_variant": variant}
    del stc

    # --- SIP variant (theta = 1, Eq. ip_flux), mixed path, same workload
    ssip = dg.Solver(mesh, P, "mixed", stream=sh, mu=1e-3, theta=1.0, C1=0.05)
    ssip.set_state(U0)
    dts = ssip.dt(0.3)
    ts, _ = timed_steps(dg, torch, ssip, dts, max(5, args.steps // 10), 2, flush, stream)
    vs = dof * 5 * len(ts) / (sum(ts) * 1e-3)
    sip_kernel = {1: "dg::stage_mixed_kernel<4, true>", 3: "dg::stage_tc_kernel<4, false, false, true>"}
    sip = {"workload": "same mesh and state, SIP (theta = 1, C1 = 0.05)", "value": vs, "unit": UNIT,
           "ms_per_step": sum(ts) / len(ts), "sip_over_iip": vs / (value / ws),
           "kernel": sip_kernel.get(ssip.variant, str(ssip.variant)), "tuned_variant": ssip.variant}
    del ssip

    # --- large variant (working set well above L2), mixed path
    large = None
    if not args.no_large:
        ml = vortex_problem(512)
        sl = dg.Solver(ml, P, "mixed", stream=sh, mu=1e-3)
        xl, yl = sl.node_coords()
        sl.set_state(dg_inputs.perturb(to_kcn(dg_inputs.isentropic_vortex(xl, yl)), seed=0))
        dtl = sl.dt(0.3)
        tl, _ = timed_steps(dg, torch, sl, dtl, max(5, args.steps // 10), 2, flush, stream)
        dofl = 4 * ml.K * NP
        vl = dofl * 5 * len(tl) / (sum(tl) * 1e-3)
        ach = algorithmic_bytes_per_step(ml.K, GEO_BYTES_MIXED) / (sum(tl) / len(tl) * 1e-3) / 1e9
        large = {"workload": "vortex p=4, 512x512 split quads", "K": ml.K, "value": vl,
                 "ms_per_step": sum(tl) / len(tl), "roofline_achieved_gbs": ach,
                 "roofline_frac": ach / peak}
        del sl

    # --- p = 6 on an 80,000-triangle O-grid (wall, far field), mixed path
    p6 = None
    if not args.no_large:
        m6 = dg_inputs.ogrid_cylinder(200, 200, 0.5, 30.0, seed=6)
        p_inf = 1.0 / (1.4 * 0.2 * 0.2)
        s6 = dg.Solver(m6, 6, "mixed", stream=sh, mu=1.0 / 150.0, rho_inf=1.0, u_inf=1.0, v_inf=0.0,
                       p_inf=p_inf)
        x6, y6 = s6.node_coords()
        U6 = to_kcn(dg_inputs.free_stream(x6.shape, rho=1.0, u=1.0, v=0.0, p=p_inf))
        U6[:, 1] *= np.tanh(4.0 * (np.hypot(x6, y6) - 0.5))
        U6[:, 3] = p_inf / 0.4 + 0.5 * U6[:, 1] ** 2 / U6[:, 0]
        s6.set_state(dg_inputs.perturb(U6, seed=3, amp=1e-3))
        dt6 = s6.dt(0.3)
        t6, _ = timed_steps(dg, torch, s6, dt6, max(5, args.steps // 10), 2, flush, stream)
        dof6 = 4 * m6.K * 28
        ach6 = (4 * m6.K * 28 * (24 + 4 * 32) + 5 * m6.K * GEO_BYTES_MIXED) / (sum(t6) / len(t6) * 1e-3) / 1e9
        p6 = {"workload": "p=6 (Np=28), seeded O-grid 200x200 (K=80,000), Re=150, M=0.2, wall + far field",
              "K": m6.K, "value": dof6 * 5 * len(t6) / (sum(t6) * 1e-3), "unit": UNIT,
              "ms_per_step": sum(t6) / len(t6), "roofline_achieved_gbs": ach6, "roofline_frac": ach6 / peak}
        del s6

    # --- batched VIV sweep: 64 cases, 10k-60k triangles, p = 3..6 (Algorithm 3 per case
    #     on the device, one CUDA graph per step), mixed path
    batch = None
    if not args.no_large:
        batch = run_batch(dg, torch, dg_inputs, to_kcn, np, peak, steps=max(10, args.steps // 50))

    # --- surrogate MLP (67 -> 3 x 128 GELU -> 2): full-batch Adam steps at B = 4096
    mlp_line = run_mlp(dg, torch, np) if not args.no_large else None

    # --- broken gradient (a2) on the tensor cores through tcgen05 against FP64
    grad_line = run_gradient(dg, torch, dg_inputs, to_kcn, peak) if not args.no_large else None

    # --- end to end through the C ABI with host buffers (pinned)
    host_in = torch.empty((K, 4, NP), dtype=torch.float64, pin_memory=True)
    host_in.copy_(torch.from_numpy(U0))
    host_out = torch.empty_like(host_in, pin_memory=True)
    e2e_steps = max(3, args.steps // 10)
    for _ in range(2):
        dg.dg_set_state(s.ctx, host_in)
        s.step(0.0, dt)
        dg.dg_get_state(s.ctx, host_out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        dg.dg_set_state(s.ctx, host_in)
        s.step(0.0, dt)
        dg.dg_get_state(s.ctx, host_out)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": ws * dof * 5 * e2e_steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(host_in.numel() * 8), "d2h_bytes_per_step": int(host_out.numel() * 8)}

    cpu = cpu1 = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(budget_s=args.cpu_seconds)
        cpu1 = cpu_baseline(budget_s=args.cpu_seconds, threads=1)

    if ws > 1:
        torch.distributed.barrier()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic: seeded isentropic vortex on a periodic square",
            "config": dict(CONFIG, parallelism=f"replicas x{ws}"),
            "roofline": roofline,
            "fp64_path": {"value": v64, "unit": UNIT, "ms_per_step": sum(t64) / len(t64),
                          "mixed_over_fp64": value / ws / v64, "roofline": roof64},
            "with_source": with_source,
            "overint_path": overint,
            "large_mesh": large,
            "fused_steps": fused,
            "sip_path": sip,
            "tensor_core_path": tc,
            "p6_large": p6,
            "batch_viv": batch,
            "mlp": mlp_line,
            "gradient": grad_line,
            "cpu_baseline": cpu,
            "cpu_baseline_1t": cpu1,
            "e2e": e2e,
            "clocks": clk.summary(),
            "gpu_launches": int(launches),
            "finite": bool(ok),
        }
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


def build_batch(dg, dg_inputs, to_kcn, np):
    """The 64-case reduced-velocity sweep as one batch solver with its seeded
    start states; returns the solver, the cases, the DOF count and the
    algorithmic bytes of one step."""
    gamma, mach = 1.4, 0.2
    p_inf = 1.0 / (gamma * mach * mach)
    sweep = dg_inputs.viv_sweep()
    cases = []
    for c in sweep:
        fn = 1.0 / c["ustar"]
        cases.append(dict(mesh=dg_inputs.sweep_mesh(c), p=c["p"], mu=1.0 / c["re"], M_r=1.0,
                          C_r=4 * np.pi * fn * c["zeta"], K_r=(1 + 1 / c["mstar"]) * (2 * np.pi * fn) ** 2,
                          mass=c["mstar"] * np.pi / 4.0))
    b = dg.BatchSolver(cases, rho_inf=1.0, u_inf=1.0, v_inf=0.0, p_inf=p_inf)
    dof, bytes_step = 0, 0
    for i, c in enumerate(cases):
        x, y = b.node_coords(i)
        U = to_kcn(dg_inputs.free_stream(x.shape, rho=1.0, u=1.0, v=0.0, p=p_inf))
        U[:, 1] *= np.tanh(4.0 * (np.hypot(x, y) - 0.5))
        U[:, 3] = p_inf / (gamma - 1) + 0.5 * U[:, 1] ** 2 / U[:, 0]
        b.set_state(i, dg_inputs.perturb(U, seed=100 + i, amp=1e-3))
        K, Np = c["mesh"].K, (c["p"] + 1) * (c["p"] + 2) // 2
        dof += 4 * K * Np
        # five stage launches, plus the time-step bound's read of the FP32 state copy
        # and pressures (20 B per node) with geometry and connectivity
        bytes_step += 4 * K * Np * (24 + 4 * 32) + 5 * K * GEO_BYTES_MIXED + K * Np * 20 + K * GEO_BYTES_MIXED
    return b, cases, dof, bytes_step


def run_batch(dg, torch, dg_inputs, to_kcn, np, peak, steps):
    """The 64-case reduced-velocity sweep advanced as one batch; CUDA events
    on the batch's stream around dg_batch_run (graph replays)."""
    b, cases, dof, bytes_step = build_batch(dg, dg_inputs, to_kcn, np)
    b.run(0.3, 3, use_graph=True)                        # warm-up, graphs captured
    ext = torch.cuda.ExternalStream(b.stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0 = b.launches
    e0.record(ext)
    b.run(0.3, steps, use_graph=True)
    e1.record(ext)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    ok = not np.any(b.rigid()[:, 9])
    launches = int(b.launches - n0)
    # the same with one cooperative launch per degree group and step
    b.set_fused(True)
    b.run(0.3, 3, use_graph=True)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(ext)
    b.run(0.3, steps, use_graph=True)
    f1.record(ext)
    f1.synchronize()
    ms_fused = f0.elapsed_time(f1)
    # ... and one cooperative launch for all degree groups per step
    b.set_fused(2)
    b.run(0.3, 3, use_graph=True)
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n1 = b.launches
    a0.record(ext)
    b.run(0.3, steps, use_graph=True)
    a1.record(ext)
    a1.synchronize()
    ms_all = a0.elapsed_time(a1)
    launches_all = int(b.launches - n1)
    ach = bytes_step * steps / (ms * 1e-3) / 1e9
    out = {"workload": "64 VIV cases (seeded O-grids, 10k-60k triangles each, 2.25 M in total, p = 3..6 "
                       "cycling, U* in [3, 8], Re in [100, 150], m* = 10, zeta = 1e-3, M = 0.2): dt, "
                       "Newmark, 5 stages and forces of every case per step, on the device, one CUDA graph "
                       "per step",
           "cases": len(cases), "dofs": dof, "steps": steps, "value": dof * 5 * steps / (ms * 1e-3),
           "unit": UNIT, "ms_per_step": ms / steps, "roofline_achieved_gbs": ach, "roofline_frac": ach / peak,
           "gpu_launches": launches, "finite": bool(ok),
           "fused_steps": {"ms_per_step": ms_fused / steps, "value": dof * 5 * steps / (ms_fused * 1e-3)},
           "single_launch": {"ms_per_step": ms_all / steps, "value": dof * 5 * steps / (ms_all * 1e-3),
                             "launches_per_step": launches_all / steps,
                             "note": "the five stages of all degree groups in one cooperative launch"}}
    del b
    return out


def run_gradient(dg, torch, dg_inputs, to_kcn, peak, n=512, calls=20):
    """The broken gradient of the benchmark's vortex state on n x n split quads
    (dg_broken_gradient, device outputs): FP64 on the CUDA cores against the
    tcgen05 kernel (split TF32 products in tensor memory, TMA-staged tiles);
    CUDA events over `calls` calls after warm-up."""
    mesh = vortex_problem(n)
    st = torch.cuda.current_stream()
    s = dg.Solver(mesh, P, "mixed", stream=st.cuda_stream, mu=1e-3)
    x, y = s.node_coords()
    s.set_state(dg_inputs.perturb(to_kcn(dg_inputs.isentropic_vortex(x, y)), seed=0))
    gx = torch.empty((mesh.K, 4, NP), dtype=torch.float64, device="cuda")
    gy = torch.empty_like(gx)
    dof = 4 * mesh.K * NP
    # read the state and the geometry record, write both gradients
    bytes_call = dof * 8 + mesh.K * 128 + 2 * dof * 8
    out = {"workload": f"broken gradient of the p=4 vortex state, {n}x{n} split quads (K={mesh.K})",
           "bytes_per_call": bytes_call}
    for impl, name in ((0, "fp64_cuda_cores"), (1, "tcgen05_tf32x3_tma")):
        for _ in range(3):
            dg.dg_broken_gradient(s.ctx, gx, gy, impl)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        for _ in range(calls):
            dg.dg_broken_gradient(s.ctx, gx, gy, impl)
        b.record(st)
        b.synchronize()
        dg.dg_barrier_status(s.ctx)
        us = a.elapsed_time(b) / calls * 1e3
        gbs = bytes_call / (us * 1e-6) / 1e9
        out[name] = {"us_per_call": us, "achieved_gbs": gbs, "frac_of_hbm": gbs / peak,
                     "dof_per_s": dof / (us * 1e-6)}
    del s
    return out


def run_mlp(dg, torch, np, B=4096, steps=200):
    """Training throughput of the surrogate network's kernels (host clock
    around dg_mlp_train, which synchronises its stream before returning)."""
    net = dg.Mlp(67, 128, 3, 2, max_batch=B, seed=0)
    rng = np.random.default_rng(0)
    X = torch.from_numpy(rng.normal(size=(B, 67)).astype(np.float32)).cuda()
    T = torch.from_numpy(rng.normal(size=(B, 2)).astype(np.float32)).cuda()
    # warm-up with the same call (same arrays and loss history): the timed
    # call replays the step graph the warm-up captured
    hist = torch.empty(steps, dtype=torch.float32, device="cuda")
    net.train(X, T, steps, 1e-3, out=hist)
    n0 = net.launches
    t0 = time.perf_counter()
    net.train(X, T, steps, 1e-3, out=hist)
    el = time.perf_counter() - t0
    macs = 67 * 128 + 2 * 128 * 128 + 128 * 2              # per sample, forward
    flops = 2 * B * macs * 3 - 2 * B * 67 * 128            # forward, weight and input gradients (none for x)
    return {"workload": "load-surrogate MLP 67 -> 3 x 128 GELU -> 2, full-batch Adam, B = 4096, bf16 MMA "
                        "with FP32 accumulation", "samples_per_s": B * steps / el, "ms_per_step": el / steps * 1e3,
            "tflops": flops * steps / el / 1e12, "launches_per_step": (net.launches - n0) / steps,
            "timing": "host clock around a synchronising call"}


def cpu_baseline(budget_s=20.0, threads=None):
    """The oracle (plain FP64 C, OpenMP over elements) on the host cores (all
    of them, or `threads`): LSRK steps of the benchmark's own p = 4 vortex
    mesh (128 x 128 split quads), as many as fit the time budget (at least
    one)."""
    import numpy as np
    import dg_inputs
    import oracle
    from dg_inputs.states import to_kcn
    oracle.build_oracle()
    cores = threads or os.cpu_count() or 1
    oracle.set_threads(cores)
    n = 128
    m = dg_inputs.periodic_square(n)
    Pq = oracle.Problem(m, P, mu=1e-3)
    U = to_kcn(dg_inputs.isentropic_vortex(Pq.x, Pq.y))
    t0 = time.perf_counter()
    U = Pq.lsrk_step(U, 0.0, 1e-5)                  # calibration step, untimed
    per_step = time.perf_counter() - t0
    steps = int(max(1, min(200, budget_s / max(per_step, 1e-6))))
    t0 = time.perf_counter()
    for _ in range(steps):
        U = Pq.lsrk_step(U, 0.0, 1e-5)
    el = time.perf_counter() - t0
    dof = 4 * m.K * NP
    return {"value": dof * 5 * steps / el, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
            "sample": f"{steps} LSRK step(s) (5 residual evaluations each) of the p=4 vortex on "
                      f"{n}x{n} split quads (K={m.K}), same method as the GPU path",
            "seconds": el}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import dg_inputs
    import oracle
    from dg_inputs.states import to_kcn
    oracle.build_oracle()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    # one step of the reference arm: one LSRK step of a bounded sample mesh,
    # sized so that warmup + steps take about a minute and a half in total
    m = dg_inputs.periodic_square(16)
    Pq = oracle.Problem(m, P, mu=1e-3)
    U = to_kcn(dg_inputs.isentropic_vortex(Pq.x, Pq.y))
    t0 = time.perf_counter()
    Pq.lsrk_step(U, 0.0, 1e-5)
    per_elem = (time.perf_counter() - t0) / m.K
    total = args.steps + args.warmup
    n = int(max(4, min(128, (90.0 / total / max(per_elem, 1e-9) / 2) ** 0.5)))
    m = dg_inputs.periodic_square(n)
    Pq = oracle.Problem(m, P, mu=1e-3)
    U = to_kcn(dg_inputs.isentropic_vortex(Pq.x, Pq.y))
    dt, _ = Pq.dt(U, 0.3)
    for _ in range(args.warmup):
        U = Pq.lsrk_step(U, 0.0, dt)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U = Pq.lsrk_step(U, 0.0, dt)
    el = time.perf_counter() - t0
    dof = 4 * m.K * NP
    value = dof * 5 * args.steps / el
    sample = (f"oracle: one LSRK step per benchmark step of the p=4 vortex on {n}x{n} split quads "
              f"(K={m.K}) on {oracle.get_threads()} host threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic: seeded isentropic vortex on a periodic square",
            "config": dict(CONFIG, parallelism="host cores, rank 0",
                           precision="FP64 throughout (the oracle)"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def strouhal(t, cl):
    """Shedding frequency (D = |v_inf| = 1) from the upward zero crossings of
    C_L - mean C_L; None with fewer than three crossings."""
    import numpy as np
    c = cl - cl.mean()
    up = np.where((c[:-1] < 0) & (c[1:] >= 0))[0]
    if len(up) < 3:
        return None
    tz = t[up] - c[up] * (t[up + 1] - t[up]) / (c[up + 1] - c[up])
    return float((len(tz) - 1) / (tz[-1] - tz[0]))


def run_config3(args):
    """Config 3: the 120 x 170 seeded O-grid (K = 40,800), p = 4, Re = 100,
    M = 0.2, from a smoothed free-stream start, `--config3-steps` steps of the
    mixed path and of the FP64 path at one fixed step (CFL `--config3-cfl` of
    the FP64 bound of the start state), C_L and C_D every 20 steps; prints
    the statistics of both histories, their largest difference (C_L relative
    to max |C_L|, C_D to mean C_D) and the wall times."""
    import numpy as np
    import torch
    import dg_inputs
    import paper_2508_17917_gb300 as dg
    from dg_inputs.states import to_kcn
    torch.cuda.set_device(0)
    gamma, mach, re = 1.4, 0.2, 100.0
    p_inf = 1.0 / (gamma * mach * mach)
    kw = dict(mu=1.0 / re, rho_inf=1.0, u_inf=1.0, v_inf=0.0, p_inf=p_inf)
    mesh = dg_inputs.ogrid_cylinder(120, 170, 0.5, 30.0, seed=0)
    sh = torch.cuda.current_stream().cuda_stream
    out, hists = {}, {}
    every = 20
    dt = None
    for prec in ("mixed", "fp64"):
        s = dg.Solver(mesh, 4, prec, stream=sh, **kw)
        x, y = s.node_coords()
        U = to_kcn(dg_inputs.free_stream(x.shape, rho=1.0, u=1.0, v=0.0, p=p_inf))
        damp = np.tanh(4.0 * (np.hypot(x, y) - 0.5))
        U[:, 1] *= damp
        U[:, 3] = p_inf / (gamma - 1) + 0.5 * U[:, 1] ** 2 / U[:, 0]
        s.set_state(dg_inputs.perturb(U, seed=0, amp=1e-3))
        if dt is None:
            s64 = dg.Solver(mesh, 4, "fp64", stream=sh, **kw)
            s64.set_state(dg_inputs.perturb(U, seed=0, amp=1e-3))
            dt = s64.dt(args.config3_cfl)
            del s64
        rows = [(0.0,) + tuple(s.wall_forces()[:2] / 0.5)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n = 0
        while n < args.config3_steps:
            k = min(every, args.config3_steps - n)
            s.steps(n * dt, dt, k)
            n += k
            F = s.wall_forces()
            rows.append((n * dt, F[0] / 0.5, F[1] / 0.5))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        h = np.array(rows)
        hists[prec] = h
        out[prec] = {"wall_s": wall, "ms_per_step_incl_forces": wall / args.config3_steps * 1e3,
                     "mean_cd": float(h[:, 1].mean()), "cd_end": float(h[-1, 1]),
                     "cl_amplitude": float(0.5 * np.ptp(h[:, 2])), "cl_end": float(h[-1, 2]),
                     "strouhal": strouhal(h[:, 0], h[:, 2]), "finite": bool(s.check_finite())}
        del s
    a, b = hists["mixed"], hists["fp64"]
    out["mixed_vs_fp64"] = {"cl": float(np.abs(a[:, 2] - b[:, 2]).max() / np.abs(b[:, 2]).max()),
                            "cd": float(np.abs(a[:, 1] - b[:, 1]).max() / np.abs(b[:, 1]).mean())}
    out.update(workload="config 3: O-grid 120x170 (K=40800), p=4, Re=100, M=0.2, smoothed free-stream start",
               steps=args.config3_steps, dt=dt, t_end=dt * args.config3_steps, cfl=args.config3_cfl,
               forces_every=every)
    if args.config3_out:
        os.makedirs(os.path.dirname(os.path.abspath(args.config3_out)), exist_ok=True)
        np.savez(args.config3_out, mixed=a, fp64=b)
    print(json.dumps(out))


def run_profile(args):
    """A few steps of one workload, for ncu captures (no timing, no extras)."""
    import torch
    import dg_inputs
    import paper_2508_17917_gb300 as dg
    from dg_inputs.states import to_kcn
    if args.profile == "batch64":
        # two steps of the 64-case sweep (the first one tunes the tile shape
        # of every degree group and captures the step graphs)
        import numpy as np
        torch.cuda.set_device(0)
        b, cases, dof, _ = build_batch(dg, dg_inputs, to_kcn, np)
        b.run(0.3, args.steps, use_graph=True)
        torch.cuda.synchronize()
        assert not np.any(b.rigid()[:, 9])
        shapes = {}
        for i, c in enumerate(cases):
            shapes.setdefault(f"p{c['p']}", b.variant(i))
        print(json.dumps({"profile": args.profile, "cases": len(cases), "dofs": dof, "steps": args.steps,
                          "launches": b.launches, "tile_shape_per_degree": shapes}))
        return
    if args.profile == "mlp4096":
        # the surrogate network's training step, replayed from its graph
        import numpy as np
        torch.cuda.set_device(0)
        B = 4096
        rng = np.random.default_rng(0)
        X = torch.from_numpy(rng.normal(size=(B, 67)).astype(np.float32)).cuda()
        T = torch.from_numpy(rng.normal(size=(B, 2)).astype(np.float32)).cuda()
        net = dg.Mlp(67, 128, 3, 2, max_batch=B, seed=0)
        hist = net.train(X, T, 12, 1e-3)
        torch.cuda.synchronize()
        assert bool(torch.isfinite(hist).all())
        print(json.dumps({"profile": args.profile, "B": B, "steps": 12, "launches": net.launches}))
        return
    if args.profile == "grad512":
        # the tcgen05 broken gradient on the 512^2 vortex state (device outputs)
        torch.cuda.set_device(0)
        mesh = vortex_problem(512)
        s = dg.Solver(mesh, P, "mixed", stream=torch.cuda.current_stream().cuda_stream, mu=1e-3)
        x, y = s.node_coords()
        s.set_state(dg_inputs.perturb(to_kcn(dg_inputs.isentropic_vortex(x, y)), seed=0))
        gx = torch.empty((mesh.K, 4, NP), dtype=torch.float64, device="cuda")
        gy = torch.empty_like(gx)
        for impl in (0, 1, 1):
            dg.dg_broken_gradient(s.ctx, gx, gy, impl)
        dg.dg_barrier_status(s.ctx)
        torch.cuda.synchronize()
        print(json.dumps({"profile": args.profile, "K": mesh.K, "launches": s.launches}))
        return
    prec, n, theta, var, p = {"mixed512": ("mixed", 512, 0.0, 0, P), "mixed128": ("mixed", 128, 0.0, 0, P),
                              "fp64_128": ("fp64", 128, 0.0, 0, P), "sip128": ("mixed", 128, 1.0, 0, P),
                              "tc512": ("mixed", 512, 0.0, 3, P), "tcsip512": ("mixed", 512, 1.0, 3, P),
                              "tc6_375": ("mixed", 375, 0.0, 3, 6)}[args.profile]
    torch.cuda.set_device(0)
    mesh = vortex_problem(n)
    s = dg.Solver(mesh, p, prec, stream=torch.cuda.current_stream().cuda_stream, mu=1e-3,
                  theta=theta, C1=0.05 if theta else 0.01)
    if var:
        s.set_variant(var)
    x, y = s.node_coords()
    s.set_state(dg_inputs.perturb(to_kcn(dg_inputs.isentropic_vortex(x, y)), seed=0))
    dt = s.dt(0.3)
    s.steps(0.0, dt, args.steps)
    torch.cuda.synchronize()
    assert s.check_finite()
    print(json.dumps({"profile": args.profile, "K": mesh.K, "steps": args.steps,
                      "launches": s.launches}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--variant", type=int, default=0, choices=[0, 1, 2, 3],
                    help="tile shape of the headline's mixed kernel (0: first-step tuner)")
    ap.add_argument("--config3", action="store_true",
                    help="long C_L / C_D histories of config 3 in both precisions (not the bench line)")
    ap.add_argument("--config3-steps", type=int, default=20000)
    ap.add_argument("--config3-cfl", type=float, default=2.0)
    ap.add_argument("--config3-out", default=None, metavar="NPZ",
                    help="also save the (t, C_D, C_L) histories of both precisions (--config3)")
    ap.add_argument("--record-traffic", default=None, metavar="CSV",
                    help="ncu raw-page CSV of one stage launch: write its DRAM bytes per DOF-stage")
    ap.add_argument("--record-k", type=int, default=2 * 512 * 512,
                    help="elements of the captured launch (--record-traffic)")
    ap.add_argument("--profile", choices=["mixed512", "mixed128", "fp64_128", "sip128", "tc512", "tcsip512", "tc6_375", "mlp4096",
                             "batch64", "grad512"], default=None)
    args = ap.parse_args()
    if args.record_traffic:
        record_traffic(args)
        return
    if args.config3:
        run_config3(args)
        return
    if args.profile:
        run_profile(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
