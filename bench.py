#!/usr/bin/env python
"""Throughput benchmark of the LES stage path: grid-point-stage updates per second.

A step is one explicit 5-stage Runge-Kutta step (all stage kernels + boundary
passes) over the whole grid; points x 5 stages x steps / time is the metric.
Default workload: the paper-scale single jet, 384x256x144 points (~14.2M),
FP64, Mach 1.4, TR 1, Re_D 1e5.  Inputs are far larger than L2 (several GB).

--impl reference times the FP64 CPU oracle (the plain C transcription of the
method) on a bounded sample of the same workload.  Under torchrun each rank
runs an independent replica of the workload (no data exchange); rank 0
prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2212_12365_gb300 import inputs as I  # noqa: E402

# Algorithmic floating-point operations per grid point and stage, counted
# from the method in the partition of the FP64 stage kernels (each point
# quantity and each interface flux once; add/sub/mul = 1, FMA = 2,
# divide/sqrt = 1, min/max/abs = 0): point pass 94 (the 5 multiplications of
# the J^-1 Q scaling included; primitives, Sutherland, spectral radii and
# lambda-bar, half point fluxes), gradients and closures 112, three interface
# fluxes 3 x 155 = 465 (the 1/2 of the interface averages of lambda-bar, mu_eff
# and kappa sits in the stored half interface J^-1), update 35: 706.  The FP32
# fused stage does the same work less the scaling, plus one J multiplication
# in the update and those three 1/2 factors per interface: 711.
FLOPS_PER_PT_STAGE = {"point": 94, "grads": 112, "iface": 465, "update": 35}
FLOPS_PER_PT_STAGE_FUSED = 711
# Algorithmic HBM bytes per point and stage: stages 2-5 read Q(l-1), Q(0) and 10
# metric values and write Q(l); stage 1 reads Q(0) once: 24 values on average.
ALGO_BYTES_PER_PT_STAGE = {"fp64": 24 * 8, "fp32": 24 * 4,
                           # separable metrics (product grids): no 3-D metric fields, 14 values
                           "fp32-sep": 14 * 4}
# DRAM bytes per point of one launch of the dominant kernel in the launch
# configuration of the run, from the ncu captures summarised in profiles/:
# keyed by workload, precision, kernel and (fused stage) the decomposition in
# use.  Each capture records the SHA-256 prefix of the kernel's source file
# at capture time; when the file has changed since, the figure no longer
# describes the kernel that runs and the lookup gives None.
_PAPER_JET = "jet-384x256x144"
KERNEL_SOURCE = {"k_iface": "les_stage.cu", "k_fused": "les_fused.cu"}
TRAFFIC_BYTES_PER_POINT = {  # (workload, precision, kernel, decomposition) -> (bytes per point, source sha16)
    # profiles/stage_kernels_fp64_jet-384x256x144.md: 13415.1 + 1682.3 MB per launch
    (_PAPER_JET, "fp64", "k_iface", None): (1066.51, "e93049f182835582"),
    # profiles/fused_stage_fp32_jet-384x256x144.md and ..._separable_...
    (_PAPER_JET, "fp32", "k_fused", "ty=16 kc=balanced"): (128.55, "2231f6aa9a29f415"),
    (_PAPER_JET, "fp32", "k_fused", "ty=16 kc=lockstep"): (106.47, "2231f6aa9a29f415"),
    (_PAPER_JET, "fp32-sep", "k_fused", "ty=16 kc=balanced"): (77.23, "2231f6aa9a29f415"),
    (_PAPER_JET, "fp32-sep", "k_fused", "ty=16 kc=lockstep"): (55.67, "2231f6aa9a29f415"),
}


def source_sha16(kname: str):
    """SHA-256 prefix of the source file that holds kernel kname."""
    import hashlib
    f = KERNEL_SOURCE.get(kname)
    if not f:
        return None
    path = os.path.join(ROOT, "paper_2212_12365_gb300", "csrc", f)
    try:
        return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]
    except OSError:
        return None


def traffic_bytes_per_point(workload: str, prec: str, kname: str, describe: str, table=None):
    """The captured DRAM bytes per point of the dominant kernel for this run's
    workload, precision and (fused stage) decomposition, read from the
    handle's description ("... ty=8 kc=lockstep ..."); None if not captured
    or if the kernel's source changed after the capture."""
    table = TRAFFIC_BYTES_PER_POINT if table is None else table
    decomp = None
    if prec != "fp64":
        mt = re.search(r"ty=(\d+) kc=(\w+)", describe)
        decomp = f"ty={mt.group(1)} kc={mt.group(2)}" if mt else None
    hit = table.get((workload, prec, kname, decomp))
    if hit is None or hit[1] != source_sha16(kname):
        return None
    return hit[0]


# Arithmetic-pipe utilisation of the dominant kernel from the committed ncu
# captures (sm__inst_executed_pipe_*, % of peak sustained while active), with
# the source hash of the captured kernel as above
PIPE_UTIL_NCU = {  # (precision, kernel) -> (metrics dict, source sha16)
    # profiles/stage_kernels_fp64_jet-384x256x144.md (192x128x72 capture)
    ("fp64", "k_iface"): ({"fp64_pipe_pct": 88.82, "executed_fp64_flop_per_point": 459.8,
                          "dadd_dmul_dfma_per_point": [118.9, 67.4, 136.8]}, "e93049f182835582"),
    # profiles/fused_stage_fp32_jet-384x256x144.md (192x128x72 capture, 32x16 tiles)
    ("fp32", "k_fused"): ({"fma_pipe_pct": 33.8, "fmaheavy_pct": 33.0, "fmalite_pct": 34.0, "issue_active_pct": 37.8,
                          "executed_fp32_flop_per_point": 1320.6, "thread_instructions_per_point": 1087.1},
                         "2231f6aa9a29f415"),
    ("fp32-sep", "k_fused"): ({"fma_pipe_pct": 32.6, "fmaheavy_pct": 34.7, "fmalite_pct": 30.1,
                              "issue_active_pct": 40.5, "executed_fp32_flop_per_point": 819.8,
                              "thread_instructions_per_point": 858.0}, "2231f6aa9a29f415"),
}
# Nominal multiply-add throughput of GB300 (unit counts x the maximum clock),
# reported beside the measured figures: 2 DFMA and 128 FFMA per clock and SM.
FP64_NOMINAL_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
HBM_NOMINAL_GBS = 7900.0  # GB300 HBM3e, nominal

def _batch64():
    jets = I.batch_jets(64, seed=4)
    return [g for g, _ in jets], [f for _, f in jets]


WORKLOADS = {
    "jet-384x256x144": (I.jet_paper_scale, "fp64"),
    "batch-64": (_batch64, "fp32"),
    "jet-768x384x192": (I.jet_large, "fp32"),
    "jet-48x32x32": (I.jet_small, "fp64"),
    "jet-192x128x72": (I.jet_medium, "fp64"),
    # the paper's polar mesh with the centerline condition (not a product grid)
    "polar-384x192x192": (I.polar_jet_paper_scale, "fp64"),
}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            parts = [p.strip() for p in l.split(",")]
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate_rate(local_ms, points_per_rank, steps, ws, device):
    """Whole-job rate of ws replicas: all ranks' point-stage updates divided by
    the slowest rank's time (max over ranks by all-reduce)."""
    ms = float(local_ms)
    if ws > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ws * points_per_rank * 5 * steps / (ms / 1e3), ms


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def host_cpu():
    """Host CPU description: architecture and model (x86 'model name', or the
    Arm implementer/part numbers)."""
    import platform
    model = None
    try:
        info = open("/proc/cpuinfo").read().splitlines()
        kv = [l.split(":", 1) for l in info if ":" in l]
        d = {}
        for k, v in kv:
            d.setdefault(k.strip(), v.strip())
        model = d.get("model name") or (f"implementer {d.get('CPU implementer')} part {d.get('CPU part')}"
                                        if "CPU part" in d else None)
    except OSError:
        pass
    return {"arch": platform.machine(), "model": model, "nproc": os.cpu_count()}


def cpu_baseline(spec, fp, budget_s=12.0, steps=1):
    """The oracle as it stands on a bounded k-slab of the workload: one RK step
    (5 stages); the slab grows until the run takes ~budget_s."""
    import oracle

    def to_oracle(sp, f):
        g = oracle.Grid(x=sp.x, y=sp.y, z=sp.z, dims=tuple(sp.dims), periodic=tuple(sp.periodic),
                        shift=np.asarray(sp.shift), bc=tuple(sp.bc))
        return g, oracle.Params(**{k: getattr(f, k) for k in oracle.Params.__dataclass_fields__})

    ni, nj, nk = spec.dims
    nplanes = 4
    best = None
    while True:
        k0 = max(0, nk // 2 - nplanes // 2)
        slab = I.jet_slab(spec, k0, k0 + nplanes)
        g, p = to_oracle(slab, fp)
        m = oracle.metrics(g)
        q = oracle.apply_bc(g, p, m, oracle.qhat_from(g, p, m, I.ambient_primitives(g.N, fp.TR), True), 0)
        dt = oracle.dt_cfl(g, p, m, q)
        t0 = time.perf_counter()
        oracle.step(g, p, m, q, steps, 0, dt)
        el = time.perf_counter() - t0
        best = (g.N * 5 * steps / el, el, nplanes)
        if el > budget_s / 4 or nplanes * 2 > nk:
            break
        nplanes *= 2
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": best[0], "unit": "grid-point-stage updates/s", "cores": cores, "kind": "oracle",
            "sample": f"{steps} RK step(s) on a {ni}x{nj}x{best[2]} k-slab of the workload "
                      f"({best[1]:.1f} s)", "cpu": host_cpu()}


def cpu_baseline_1core(workload, budget_s=4.0):
    """The same oracle sample on one host core (OpenMP limited to one thread in
    a child process; it touches no GPU)."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "spec, fp = bench.WORKLOADS[%r][0](); "
            "print(json.dumps(bench.cpu_baseline(spec, fp, budget_s=%r)))" % (ROOT, workload, budget_s))
    env = dict(os.environ, OMP_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                             timeout=300, check=True).stdout
        return json.loads(out.strip().splitlines()[-1])
    except Exception:
        return None


def workload_config(args, prec, specs, fps, batch, ws, probe=None):
    """The JSON line's config object (the same for both arms of a workload)."""
    return {"workload": args.workload, "precision": prec, "points": sum(g.N for g in specs),
            "grid": [list(g.dims) for g in specs] if batch else list(specs[0].dims),
            "jets": len(specs),
            "mach_j": [f.mach_j for f in fps] if batch else fps[0].mach_j,
            "TR": [round(f.TR, 3) for f in fps] if batch else fps[0].TR,
            "Re_D": [round(f.Re) for f in fps] if batch else fps[0].Re,
            "tiling": args.tiling,
            "probe": probe,
            "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
            "l2": "inputs larger than L2 (state + metrics + scratch are GBs)"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    make, prec_default = WORKLOADS[args.workload]
    prec = args.precision or prec_default
    spec, fp = make()
    batch = isinstance(spec, list)
    cfg = workload_config(args, prec, spec if batch else [spec], fp if batch else [fp], batch, ws,
                          None if not (args.probe or args.workload == "jet-768x384x192") else
                          {"points": 256 * 384, "every": 5, "frames": None})
    if batch:  # a batch: the oracle samples its first jet
        spec, fp = spec[0], fp[0]
    import oracle  # noqa: F401
    oracle.build()
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(spec, fp, budget_s=4.0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(spec, fp, budget_s=8.0))
    el = time.perf_counter() - t0
    v = float(np.median([c["value"] for c in vals]))
    line = {"impl": "reference", "metric": "grid-point-stage updates/s", "value": v,
            "unit": "grid-point-stage updates/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {**vals[0], "value": v},
            "e2e": {"value": v, "unit": "grid-point-stage updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def hbm_peak_gbs():
    """HBM denominator: the measured copy bandwidth of this machine's
    GB300s, or the profiling recipe's fallback figure when that file is
    missing (labelled as such)."""
    v = measured_peaks().get("hbm_gbs")
    if v:
        return float(v), "measured (MEASURED_PEAKS.json, copy bandwidth)"
    return 6800.0, "fallback 6.8 TB/s (MEASURED_PEAKS.json missing)"


_ALU = {}


def alu_peaks(les):
    """Measured multiply-add throughput of this GPU (TFLOP/s): FP64 DFMA, FP32
    FFMA and paired FP32 (fma.rn.f32x2), each a short independent-chain loop
    timed with CUDA events (les_measure_peak); measured once per process."""
    if not _ALU:
        _ALU["fp64_fma"] = les.les_measure_peak(les.LES_PEAK_FP64_FMA)
        _ALU["fp32_fma"] = les.les_measure_peak(les.LES_PEAK_FP32_FMA)
        _ALU["fp32x2_fma"] = les.les_measure_peak(les.LES_PEAK_FP32X2_FMA)
    return dict(_ALU)


def _time_steps(solver, steps, torch):
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    solver.step(steps)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def batched_form(args, les, torch, fp64_value):
    """The batched form (64 jets of uneven grids, Mach, temperature ratio,
    Reynolds number and seed, one persistent launch per stage, the step a
    CUDA graph), FP32 and FP32 with separable metrics: device rate after the
    warm-up, the HBM fraction of the algorithmic bytes, and a bit-for-bit
    check of three jets against single-jet handles after the same steps."""
    specs, fps = _batch64()
    N = sum(g.N for g in specs)
    hbm, _ = hbm_peak_gbs()
    out = {"jets": len(specs), "points": N}
    check_jets = (0, len(specs) // 2, len(specs) - 1)
    nchk = 3
    for name, P in (("fp32", les.LES_FP32), ("fp32-sep", les.LES_FP32_SEPARABLE)):
        b = les.Solver(specs, fps, P)
        for j, (g, f) in enumerate(zip(specs, fps)):
            b.set_state(I.ambient_primitives(g.N, f.TR), les.LES_STATE_PRIMITIVE, jet=j)
        b.step(nchk)
        same = True
        for j in check_jets:
            s1 = les.Solver(specs[j], fps[j], P)
            s1.set_state(I.ambient_primitives(specs[j].N, fps[j].TR), les.LES_STATE_PRIMITIVE)
            s1.step(nchk)
            same = same and bool(np.array_equal(s1.get_state(les.LES_STATE_RAW),
                                                b.get_state(les.LES_STATE_RAW, jet=j)))
            s1.close()
        b.step(args.warmup)
        ms = _time_steps(b, args.steps, torch)
        v = N * 5 * args.steps / (ms / 1e3)
        out[name] = {"value": v, "ms_per_step": ms / args.steps, "speedup_vs_fp64_single_jet": v / fp64_value,
                     "hbm_frac_algorithmic": v * ALGO_BYTES_PER_PT_STAGE[name] / 1e9 / hbm,
                     "bit_identical_to_single_jets": {"jets": list(check_jets), "after_steps": nchk,
                                                      "equal": same},
                     "stage": les.les_describe(b.h)}
        b.close()
    return out


def large_probe_form(args, les, torch):
    """The large FP32 run: 768x384x192 (56.6 M points), Mach 1.4, temperature
    ratio 2, with the cylinder surface probe (r = 3D, 256 x 384 points, every
    5 steps) written to a device ring inside the captured step."""
    spec, fp = I.jet_large()
    s = les.Solver(spec, fp, les.LES_FP32)
    s.set_state(I.ambient_primitives(spec.N, fp.TR), les.LES_STATE_PRIMITIVE)
    xyz = I.cylinder_points(3.0, 256, 384, 0.5, spec.x.max() - 0.5)
    cap = 64
    ring = torch.zeros((cap, 5, xyz.shape[1]), device="cuda", dtype=torch.float32)
    les.les_probe_surface(s.h, xyz, 5, ring.data_ptr(), cap)
    s.step(args.warmup)
    ms = _time_steps(s, args.steps, torch)
    v = spec.N * 5 * args.steps / (ms / 1e3)
    frames = les.les_probe_frames(s.h)
    hbm, _ = hbm_peak_gbs()
    out = {"workload": "jet-768x384x192", "precision": "fp32", "points": spec.N, "value": v,
           "ms_per_step": ms / args.steps,
           "hbm_frac_algorithmic": v * ALGO_BYTES_PER_PT_STAGE["fp32"] / 1e9 / hbm,
           "probe": {"points": int(xyz.shape[1]), "every": 5, "frames": int(frames),
                     "finite": bool(torch.isfinite(ring).all().item())},
           "stage": les.les_describe(s.h)}
    s.close()
    return out


# FP32 operations per (panel, observer, time) evaluation of the FW-H observer
# pass: emission-frame position 2, seven retarded interpolations 21, the two
# radial projections 10, the integrand 5, the compensated sum 4.
FWH_FLOP_PER_EVAL = 42


def fwh_form(les, torch, alu):
    """FW-H far-field pressure (les_fwh) on the large jet's probe surface
    (r = 3D, 256 azimuths x 384 axial stations over x = 0.5..29.5): 1024
    synthetic FP32 frames (four seeded monopoles on the jet axis radiating
    Gaussian pulses into the ambient of temperature ratio 2, so the data are
    an exact acoustic field), 64 microphones on an arc of radius 60D about
    x = 15D from 20 to 120 degrees, 512 observer times.  Device time of the
    observer pass per evaluation, its FP32 FLOP rate against the measured
    FFMA peak, and the oracle's rate on a bounded sample (the CPU baseline;
    parity is the tests' business)."""
    from oracle import fwh as ofwh
    TR = 2.0
    c0, rho0, p0 = (1.0 / TR) ** 0.5, TR, 1.0 / 1.4
    xyz, nrm, area = I.cylinder_panels(3.0, 256, 384, 0.5, 29.5)
    obs = I.observer_arc(60.0, 64, 15.0)
    nfr, dtau, nt, dt_obs = 1024, 0.1, 512, 0.1
    rng = np.random.default_rng(2212)
    src_x = rng.uniform(3.0, 25.0, 4)
    t_c = rng.uniform(20.0, 60.0, 4)
    amp = rng.uniform(0.05, 0.2, 4)
    dev = torch.device("cuda")
    P = torch.tensor(xyz, dtype=torch.float64, device=dev)
    ring = torch.empty((nfr, 5, xyz.shape[1]), dtype=torch.float32, device=dev)
    sig = 1.5
    for m in range(nfr):
        t = m * dtau
        p = torch.zeros(xyz.shape[1], dtype=torch.float64, device=dev)
        u = torch.zeros((3, xyz.shape[1]), dtype=torch.float64, device=dev)
        for s_, (sx, tc, a) in enumerate(zip(src_x, t_c, amp)):
            d = P.clone()
            d[0] -= sx
            R = torch.sqrt((d * d).sum(dim=0))
            tr = t - R / c0
            q = a * torch.exp(-((tr - tc) / sig) ** 2)
            qd = -2.0 * (tr - tc) / sig ** 2 * q
            p += rho0 * qd / (4 * np.pi * R)
            u += (qd / (4 * np.pi * c0 * R) + q / (4 * np.pi * R * R)) * d / R
        ring[m, 0] = (rho0 + p / c0 ** 2).float()
        ring[m, 1:4] = u.float()
        ring[m, 4] = (p0 + p).float()
    d = obs[:, :, None] - xyz[:, None, :]
    r = np.sqrt((d * d).sum(axis=0))
    t0 = r.max() / c0 + 0.05
    assert t0 + (nt - 1) * dt_obs - r.min() / c0 <= (nfr - 1) * dtau
    torch.cuda.synchronize()
    les.les_fwh(ring.data_ptr(), les.LES_FP32, nfr, nfr, xyz, nrm, area, dtau, p0, c0, obs, t0, dt_obs, nt)
    t_wall = time.perf_counter()
    out, ms = les.les_fwh(ring.data_ptr(), les.LES_FP32, nfr, nfr, xyz, nrm, area, dtau, p0, c0, obs, t0, dt_obs,
                          nt, timings=True)
    t_wall = time.perf_counter() - t_wall
    evals = float(xyz.shape[1]) * obs.shape[1] * nt
    tflops = evals * FWH_FLOP_PER_EVAL / (ms[1] * 1e-3) / 1e12
    # CPU baseline: the oracle on a bounded sample of the same evaluation
    # (every 16th panel, one microphone, 24 observer times)
    sub = np.arange(0, xyz.shape[1], 16)
    host = ring[:, :, sub].double().cpu().numpy()
    t_cpu = time.perf_counter()
    ofwh.pressure(host, xyz[:, sub], nrm[:, sub], area[sub], dtau, rho0, p0, c0, obs[:, 32:33], t0, dt_obs * 21, 24)
    t_cpu = time.perf_counter() - t_cpu
    return {"metric": "FW-H panel-observer-time evaluations/s", "value": evals / (ms[1] * 1e-3),
            "panels": int(xyz.shape[1]), "frames": nfr, "observers": int(obs.shape[1]), "times": nt,
            "ms_source_pass": float(ms[0]), "ms_observer_pass": float(ms[1]), "wall_s_call": t_wall,
            "roofline": {"bound": "alu", "achieved": tflops, "peak": alu["fp32_fma"], "unit": "TFLOP/s",
                         "frac": tflops / alu["fp32_fma"], "flop_per_eval": FWH_FLOP_PER_EVAL,
                         "peak_source": "measured: FFMA loop of les_measure_peak on this GPU (CUDA events)"},
            "cpu_baseline": {"value": len(sub) * 24 / t_cpu, "unit": "panel-observer-time evaluations/s",
                             "cores": 1, "kind": "oracle",
                             "sample": f"{len(sub)} panels (every 16th) x 1 microphone x 24 times, numpy"},
            "p_rms_over_p0": float(np.sqrt((out ** 2).mean()) / p0)}


def precision_form(args, spec, fp, les, torch, fp64_value):
    """FP32 storage/arithmetic on the same grid (metrics and sums in FP64): its
    rate, speedup over the FP64 path, and relative L2 per field against the FP64
    path after 100 steps from the ambient start (the accuracy criterion of the
    FP32 form; more if the timed run is longer)."""
    forms = {}
    states = {}
    steps = max(100, args.warmup + args.steps)
    names = {les.LES_FP32: "fp32", les.LES_FP32_SEPARABLE: "fp32-sep"}
    for prec in (les.LES_FP32, les.LES_FP32_SEPARABLE, les.LES_FP64):
        s = les.Solver(spec, fp, prec)
        s.set_state(I.ambient_primitives(spec.N, fp.TR), les.LES_STATE_PRIMITIVE)
        if prec != les.LES_FP64:
            s.step(args.warmup)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            st = torch.cuda.current_stream()
            e0.record(st)
            s.step(args.steps)
            e1.record(st)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            forms[prec] = {"precision": names[prec], "value": spec.N * 5 * args.steps / (ms / 1e3),
                           "ms_per_step": ms / args.steps, "stage": les.les_describe(s.h)}
            s.step(steps - args.warmup - args.steps)
        else:
            s.step(steps)
        states[prec] = s.get_state(les.LES_STATE_CONSERVED)
        s.close()
    b = states[les.LES_FP64]
    for prec, f in forms.items():
        a = states[prec]
        err = np.sqrt(((a - b) ** 2).sum(axis=1) / np.maximum((b ** 2).sum(axis=1), 1e-300))
        f["speedup_vs_fp64"] = f["value"] / fp64_value
        f["rel_l2_vs_fp64_per_field"] = [float(e) for e in err]
        f["after_steps"] = steps
        f["hbm_frac_algorithmic"] = f["value"] * ALGO_BYTES_PER_PT_STAGE[names[prec]] / 1e9 / hbm_peak_gbs()[0]
    out = forms[les.LES_FP32]
    # the separable-metric stage (Cartesian-product grids only), reported apart
    out["separable"] = forms[les.LES_FP32_SEPARABLE]
    return out


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2212_12365_gb300 import build, les
    build.build()
    make, prec_default = WORKLOADS[args.workload]
    prec = args.precision or prec_default
    P = {"fp64": les.LES_FP64, "fp32": les.LES_FP32, "fp32-sep": les.LES_FP32_SEPARABLE}[prec]
    spec, fp = make()
    batch = isinstance(spec, list)
    specs = spec if batch else [spec]
    fps = fp if batch else [fp]
    for f in fps:
        f.seed = f.seed + 1000 * rank
    N = sum(g.N for g in specs)
    stream = torch.cuda.current_stream()
    solver = les.Solver(specs if batch else spec, fps if batch else fp, P,
                        stream=les.ctypes.c_void_p(stream.cuda_stream))
    for j, (g, f) in enumerate(zip(specs, fps)):
        solver.set_state(I.ambient_primitives(g.N, f.TR), les.LES_STATE_PRIMITIVE, jet=j)
    if args.tiling and P != les.LES_FP64:
        ty, kc = (int(v) for v in args.tiling.split(","))
        les.les_set_fused_tiling(solver.h, ty, kc)
    probe = None
    if args.probe or args.workload == "jet-768x384x192":
        # cylinder r = 3D, 256 azimuths x 384 axial stations, every 5 steps
        xyz = I.cylinder_points(3.0, 256, 384, 0.5, specs[0].x.max() - 0.5)
        cap = 64
        probe = torch.zeros((cap, 5, xyz.shape[1]), device="cuda",
                            dtype=torch.float64 if P == les.LES_FP64 else torch.float32)
        les.les_probe_surface(solver.h, xyz, 5, probe.data_ptr(), cap)
    # a developed state: march the start-up before timing
    solver.step(args.warmup)
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # one event per step boundary (the steps run back to back; the events
    # only give the per-step spread)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier()
    with ClockSampler(local) as clk:
        evs[0].record(stream)
        for i in range(args.steps):
            solver.step(1)
            evs[i + 1].record(stream)
        barrier()
    launches = les.les_last_launch_count(solver.h) * args.steps
    value, ms = aggregate_rate(evs[0].elapsed_time(evs[-1]), N, args.steps, ws, "cuda")
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]

    # per-kernel device time of the same stage sequence, eager with events
    prof = les.les_profile_step(solver.h, max(1, min(args.steps, 3)))
    tot = sum(v[0] for v in prof.values())
    alu = alu_peaks(les)
    if prec == "fp64":
        dom = max(FLOPS_PER_PT_STAGE, key=lambda k: prof[k][0])
        kname, flops_pt = f"k_{dom}", FLOPS_PER_PT_STAGE[dom]
        peak, peak_nominal = alu["fp64_fma"], FP64_NOMINAL_TFLOPS
        peak_source = "measured: DFMA loop of les_measure_peak on this GPU (CUDA events)"
    else:
        dom = "iface"  # the fused single-pass stage kernel is traced under this kind
        kname, flops_pt = "k_fused", FLOPS_PER_PT_STAGE_FUSED
        peak, peak_nominal = alu["fp32_fma"], FP32_NOMINAL_TFLOPS
        peak_source = "measured: FFMA loop of les_measure_peak on this GPU (CUDA events)"
    t_launch = prof[dom][0] / max(prof[dom][1], 1) / 1e3  # s per launch
    achieved = flops_pt * N / t_launch / 1e12
    hbm_peak, hbm_source = hbm_peak_gbs()
    traffic_pt = traffic_bytes_per_point(args.workload, prec, kname, les.les_describe(solver.h))
    pipe = PIPE_UTIL_NCU.get((prec, kname))
    bytes_pt_stage = ALGO_BYTES_PER_PT_STAGE[prec]
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic_pt * N if traffic_pt else None,
                "pipe_util_ncu": pipe[0] if pipe and pipe[1] == source_sha16(kname) else None,
                "peak_source": peak_source,
                "peak_nominal": peak_nominal, "frac_nominal": achieved / peak_nominal,
                "measured_alu_peaks_tflops": alu,
                "flops_per_point_stage": flops_pt,
                "share": prof[dom][0] / tot if tot else None,
                "per_kernel_ms_per_launch": {k: v[0] / max(v[1], 1) for k, v in prof.items() if v[1]},
                "stage": les.les_describe(solver.h),
                "source_sha16": source_sha16(kname),
                # the metric's "% HBM roofline": algorithmic bytes of a stage at the achieved rate
                "hbm_view": {"algorithmic_bytes_per_point_stage": bytes_pt_stage,
                             "achieved_gbs": value * bytes_pt_stage / 1e9 / ws,
                             "peak_gbs": hbm_peak, "peak_source": hbm_source,
                             "frac": value * bytes_pt_stage / 1e9 / ws / hbm_peak,
                             "frac_nominal": value * bytes_pt_stage / 1e9 / ws / HBM_NOMINAL_GBS,
                             # DRAM bytes of the dominant kernel (ncu capture) over its event-timed launch
                             "dominant_kernel_dram_gbs": traffic_pt * N / t_launch / 1e9 if traffic_pt else None}}

    # end to end through the public API: pinned host state in, step, state out
    e2e = None
    if not args.no_e2e and ws == 1 and not batch:
        host_in = torch.empty((5, N), dtype=torch.float64, pin_memory=True)
        host_out = torch.empty((5, N), dtype=torch.float64, pin_memory=True)
        host_in.numpy()[:] = solver.get_state(les.LES_STATE_RAW)
        ke = max(2, min(args.steps, 5))
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(ke):
            les._check(solver.h, les.lib().les_set_state_jet(solver.h, 0, les._dptr(host_in.numpy()),
                                                             les.LES_STATE_RAW))
            solver.step(1)
            les._check(solver.h, les.lib().les_get_state_jet(solver.h, 0, les._dptr(host_out.numpy()),
                                                             les.LES_STATE_RAW))
        ev1.record(stream)
        torch.cuda.synchronize()
        ems = ev0.elapsed_time(ev1)
        e2e = {"value": N * 5 * ke / (ems / 1e3), "unit": "grid-point-stage updates/s",
               "h2d_bytes_per_step": 5 * N * 8, "d2h_bytes_per_step": 5 * N * 8, "steps": ke}

    cpu = None
    # (a k-slab of a polar mesh would cut its azimuthal period: no CPU sample there)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and not batch and not spec.periodic[2]:
        cpu = cpu_baseline(spec, fp)
        one = cpu_baseline_1core(args.workload)
        if one:
            cpu["value_1core"] = one["value"]
            cpu["sample_1core"] = one["sample"] + ", 1 thread"
    secondary = batched = large = fwh_line = None
    default_run = rank == 0 and ws == 1 and args.workload == "jet-384x256x144" and prec == "fp64"
    if default_run and not args.no_fp32:
        secondary = precision_form(args, spec, fp, les, torch, value)
    if default_run and not args.no_extra:
        solver.close()
        solver = None
        batched = batched_form(args, les, torch, value)
        large = large_probe_form(args, les, torch)
        fwh_line = fwh_form(les, torch, alu)

    if rank == 0:
        line = {"metric": "grid-point-stage updates/s", "value": value,
                "unit": "grid-point-stage updates/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "step_ms": {"best": min(step_ms), "median": float(np.median(step_ms)), "max": max(step_ms)},
                "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32",
                "data": "synthetic",
                "config": workload_config(args, prec, specs, fps, batch, ws,
                                          None if probe is None else
                                          {"points": int(probe.shape[2]), "every": 5,
                                           "frames": les.les_probe_frames(solver.h)}),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "precision_form": secondary,
                "batched": batched,
                "large_probe": large,
                "fwh": fwh_line,
                "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    if solver is not None:
        solver.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# the paper's ten meshes (n_xi axial, n_eta radial, n_zeta azimuthal; Table
# "Mesh information"), run here as tanh-refined polar jet meshes of 30D x 12D
PAPER_MESHES = [(200, 150, 40), (400, 150, 40), (800, 150, 40), (400, 75, 40), (400, 300, 40),
                (400, 150, 10), (400, 150, 60), (800, 300, 120), (200, 75, 40), (200, 75, 20)]


def run_sweep(args):
    """Throughput over the paper's mesh sizes, FP64 and FP32, one JSON line
    ({"sweep": [...]}): per mesh the device rate of `steps` timed steps after
    `warmup` steps from the ambient start (CUDA events on the solver's
    stream)."""
    import torch
    torch.cuda.set_device(0)
    from paper_2212_12365_gb300 import build, les
    build.build()
    stream = torch.cuda.current_stream()
    rows = []
    for n, dims in enumerate(PAPER_MESHES, start=1):
        spec = I.polar_jet_grid(*dims, 30.0, 12.0)
        fp = I.FlowParams(seed=n)
        row = {"mesh": n, "dims": list(dims), "points": spec.N}
        for name, P in (("fp64", les.LES_FP64), ("fp32", les.LES_FP32)):
            s = les.Solver(spec, fp, P, stream=les.ctypes.c_void_p(stream.cuda_stream))
            s.set_state(I.ambient_primitives(spec.N, fp.TR), les.LES_STATE_PRIMITIVE)
            s.step(args.warmup)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step(args.steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            row[name] = {"value": spec.N * 5 / (ms / 1e3), "ms_per_step": ms, "stage": les.les_describe(s.h)}
            s.close()
        rows.append(row)
    print(json.dumps({"metric": "grid-point-stage updates/s", "unit": "grid-point-stage updates/s",
                      "data": "synthetic", "sweep": rows}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="jet-384x256x144", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default=None, choices=["fp64", "fp32", "fp32-sep"],
                    help="fp32-sep: FP32 with the separable-metric stage (product grids)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp32", action="store_true", help="skip the FP32 line of the FP64 default run")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the batched (64 jets) and large probed (768x384x192) keys of the default run")
    ap.add_argument("--probe", action="store_true", help="register the cylinder surface probe")
    ap.add_argument("--tiling", default=None,
                    help="TY,KC: fix the fused FP32 stage's tile height and k-chunk (0 = balanced, -1 = lockstep) "
                         "instead of autotuning")
    ap.add_argument("--sweep", action="store_true",
                    help="throughput over the paper's ten mesh sizes (polar meshes), FP64 and FP32")
    ap.add_argument("--fwh", action="store_true",
                    help="only the FW-H far-field evaluation of the default run's 'fwh' key (one JSON line)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.sweep:
        run_sweep(args)
    elif args.fwh:
        import torch
        from paper_2212_12365_gb300 import build, les
        build.build()
        torch.cuda.set_device(0)
        print(json.dumps(fwh_form(les, torch, alu_peaks(les))), flush=True)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
