"""Throughput of the fused finite-volume residual + RK stage on GB300.

Metric: Gcell-updates/s per RK stage (cells x stages / s) on the 3D
manufactured-solution block, 128^3 perturbed-curvilinear cells, FP64 state,
MUSCL + van Leer + Roe, 4-stage RK (the synthetic stand-in for the paper's
cases; Section 8 cases' grids are not available), in plain binary64
arithmetic.  One step = one full RK step: per stage the ghost fill and the
fused residual + update kernel.

Printed (rank 0): one JSON line per variant workload / form and one for the
adjoint workload, then LAST the short headline line.  Its ``forms`` list
reports the double-float and binary32-flux forms and the batched multi-block
workload against the binary64 line, with each form's error against the
binary64 path (one residual; and the binary32-flux form's drift after 100
stages).  ``--impl reference`` times the CPU oracle (the only other place
this file runs oracle code) on a bounded sample of the same workload;
``--peaks`` prints the measured arithmetic rates only.
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
sys.path.insert(0, ROOT)

import cases  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
# Unit counts and clocks of the GB300 (152 SMs, 128 FP32 lanes per SM,
# 2070 MHz maximum SM clock) and its nominal FP64 rate (1.25 TFLOP/s).
N_SM, FP32_LANES, SM_HZ = 152, 128, 2.07e9
FP64_NOMINAL_FLOPS = 1.25e12
# Algorithmic FP64 operations of one face with the default method (van Leer,
# kappa = -1, Harten fix), as the oracle's op-counting scalar counts them
# (add/sub, mul, div, sqrt, abs); tests/test_bench_constants.py checks them.
FACE_OPS = {"add": 153, "mul": 162, "div": 50, "sqrt": 3, "abs": 23}
# per interior cell beyond its faces: primitive recovery 12, fixed-order sums
# with the source 35, RK update 11
CELL_OPS = 58
# binary32 instructions of one double-float operation (fv_arith.cuh): sloppy
# add 11, double-float product 7, quotient 27, square root 25, |x| 2
DF64_COST = {"add": 11, "mul": 7, "div": 27, "sqrt": 25, "abs": 2}


# one viscous face (the oracle's own count: face gradients of u, v, w, T,
# stresses, heat flux, flux; constant viscosity) and, per cell, the viscous
# pair differences of the 4 momentum/energy components
VISC_FACE_OPS = {"add": 82, "mul": 89, "div": 24, "sqrt": 0, "abs": 0}


def alu_ops_per_cell(dim: int = 3, visc: bool = False) -> int:
    n = dim * sum(FACE_OPS.values()) + CELL_OPS
    if visc:
        n += dim * sum(VISC_FACE_OPS.values()) + 8 * dim
    return n


def alu_peak(precision: str, rates: dict):
    """Measured FP64-operation roofline of the arithmetic forms and how it
    was obtained.  binary64: twice the measured binary64 FMA rate (FLOP/s,
    an FMA counted as two operations).  double-float: the measured rate of
    the face's operation mix, sum_k n_k / sum_k (n_k / rate_k) over the
    oracle's per-face counts n_k of add, multiply, divide, square root and
    absolute value and the measured double-float rate of each."""
    if precision == "fp64":
        return 2.0 * rates["fp64_fma"], "measured: 2 x binary64 FMA rate (fv_probe_alu_rates)"
    key = {"add": "df64_add", "mul": "df64_mul", "div": "df64_div", "sqrt": "df64_sqrt", "abs": "df64_abs"}
    t = sum(FACE_OPS[k] / rates[key[k]] for k in FACE_OPS)
    return sum(FACE_OPS.values()) / t, "measured: double-float rates over the face's operation mix"


def nominal_alu_peak(precision: str) -> float:
    """Unit-count estimate, for context beside the measured peak: the
    nominal FP64 rate, or the FP32 lane rate over the mean binary32 cost of
    one emulated operation in the face's mix."""
    if precision == "fp64":
        return FP64_NOMINAL_FLOPS
    mix = sum(FACE_OPS[k] * DF64_COST[k] for k in FACE_OPS) / sum(FACE_OPS.values())
    return N_SM * FP32_LANES * SM_HZ / mix


def workload(name: str):
    """Benchmark workloads; a suffix '+vl' or '+sw' selects the van Leer or
    Steger-Warming face flux instead of Roe."""
    if "+" in name:
        base, suf = name.split("+", 1)
        if suf == "ns":
            return workload_ns(base)
        pb = workload(base)
        pb.params["flux"] = {"vl": 1, "sw": 2}[suf]
        pb.name += "_" + {"vl": "vanleer_fvs", "sw": "steger_warming"}[suf]
        return pb
    if name == "mms128":
        return cases.mms_3d(128, curvilinear=True)
    if name == "large":
        return cases.large_periodic(512, 512, 256)
    if name == "multiblock":
        return cases.multiblock_batched()
    if name == "vortex":
        return cases.vortex_2d(64)
    if name == "inlet":       # the paper's largest inlet grids are ~7 M cells
        return cases.inlet_2d(4096, 1536)
    if name == "ogrid":       # wing-sized (4.2 M cells) extruded O-grid
        return cases.ellipse_ogrid(512, 128, 64)
    if name.startswith("mms"):
        return cases.mms_3d(int(name[3:]), curvilinear=True)
    raise SystemExit("unknown workload " + name)


def workload_ns(base: str):
    """Laminar Navier-Stokes versions: the manufactured 128^3 block with its
    viscous source (mu = 0.05), or the extruded O-grid with adiabatic no-slip
    walls and air's Sutherland viscosity (SI units)."""
    if base.startswith("mms"):
        n = 128 if base == "mms128" else int(base[3:])
        return cases.mms_3d(n, curvilinear=True, visc=1, mu=0.05)
    pb = workload(base)
    pb.params.update(visc=1, mu=1.716e-5, sutherland=1, t_ref=273.15, s_suth=110.4, r_gas=287.0)
    pb.bcs = [cases.BCPatch(p.block, p.face, p.lo, p.hi,
                            cases.BC_NOSLIP_WALL if p.kind == cases.BC_SLIP_WALL else p.kind, p.state)
              for p in pb.bcs]
    pb.name += "_ns"
    return pb


def algorithmic_bytes(pb, stage: int, curvilinear: bool, precision: str = "fp64") -> float:
    """Bytes a cell-update must move at least: read Q^(m-1) (40 B), read Q^(0)
    for stages > 1 (40 B), write Q^(m) (40 B); curvilinear metrics - the face
    vector of each face family (3 in 3D, 2 in 2D) in the form's storage, 24 B
    (binary64, or a pair of binary32 per value) or 12 B (the binary32-flux
    form) - and 8 B of 1/Omega; a source term 40 B; exchanged ghost cells
    read and write 80 B each; a physical boundary position writes its two
    ghost layers and reads one interior cell (120 B)."""
    n = pb.ncells
    per = 80.0 + (40.0 if stage > 1 else 0.0)
    if curvilinear:
        per += (12.0 if precision == "fp32flux" else 24.0) * pb.dim + 8.0
    if pb.source is not None:
        per += 40.0
    if pb.params.get("visc", 0):
        per += 80.0          # the auxiliary-volume geometry (Omega + 3 face vectors) read once
    ghosts = 0
    for c in pb.conns:
        ghosts += 2 * (c.dst_hi[0] - c.dst_lo[0]) * (c.dst_hi[1] - c.dst_lo[1])
    bc = sum((p.hi[0] - p.lo[0]) * (p.hi[1] - p.lo[1]) for p in getattr(pb, "bcs", []) or [])
    return per * n + 80.0 * ghosts + 120.0 * bc


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return FALLBACK_PEAKS, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        # one long-lived nvidia-smi in loop mode (a sample every 100 ms); a
        # process per sample would take longer than the timed region
        try:
            self._p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                        "--format=csv,noheader,nounits", "-lms", "100"],
                                       stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            return
        for line in self._p.stdout:
            row = [x.strip() for x in line.strip().split(",")]
            if len(row) >= 7:
                self.rows.append(row)
            if self._stop.is_set():
                break

    def __enter__(self):
        self._p = None
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        time.sleep(0.3)     # let the first sample land before the region starts
        return self

    def __exit__(self, *a):
        time.sleep(0.15)    # one more sample at the end of the region
        self._stop.set()
        if self._p is not None:
            self._p.terminate()
            try:
                self._p.wait(timeout=5)
            except Exception:
                self._p.kill()
        if self._t:
            self._t.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for n, v in zip(names, r[3:7]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def kernel_hash() -> str:
    """Hash of the sources the fused stage kernel is compiled from (its
    template, face code, arithmetic, shared structures and the translation
    units instantiating it): the traffic measured for it is valid while this
    is unchanged."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2012_02925_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f in ("fv_stage.cuh", "fv_face.cuh", "fv_arith.cuh", "fv_viscface.cuh", "fv_internal.h") or \
                (f.startswith("fv_stage_") and f.endswith(".cu")):
            h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def load_traffic():
    """DRAM traffic per launch from a committed ncu summary, valid only for the
    kernel sources it was captured from."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            t = json.load(f)
    except Exception:
        return {}
    return t if t.get("kernel_hash") == kernel_hash() else {}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def make_solver(pb, precision, tile=0, kchunk=0, tune=True, reps=3):
    import torch
    import paper_2012_02925_gb300 as fv
    s = fv.Solver.from_problem(pb, precision=precision, tile=tile, kchunk=kchunk)
    s.set_state(torch.from_numpy(pb.q).cuda())
    if pb.source is not None:
        s.set_source(torch.from_numpy(np.concatenate([x.ravel() for x in pb.source])).cuda())
    if tune and tile == 0:
        s.autotune(pb.dt, reps=reps)
    torch.cuda.synchronize()
    return s


def time_steps(s, pb, steps, warmup, use_graph=True, per_step=None):
    """Device time of `steps` RK steps (CUDA events on the launching stream);
    with a list `per_step`, an event after every step also gives each step's
    time (the repeats whose spread is reported)."""
    import torch
    for _ in range(warmup):
        s.rk_step(pb.dt, use_graph=use_graph)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1 if per_step is not None else 2)]
    ev[0].record(st)
    for n in range(steps):
        s.rk_step(pb.dt, use_graph=use_graph)
        if per_step is not None:
            ev[n + 1].record(st)
    ev[-1].record(st)
    torch.cuda.synchronize()
    if per_step is not None:
        per_step.extend(ev[n].elapsed_time(ev[n + 1]) for n in range(steps))
    return ev[0].elapsed_time(ev[-1]) / 1e3


def time_stage_kernels(s, pb, reps):
    """Average device time of each RK stage launch (exchange + fused kernel)
    and of the exchange alone, CUDA events on the launching stream."""
    import torch
    st = torch.cuda.current_stream()
    M = s.n_stages
    out = []
    for m in range(1, M + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.rk_stage(m, pb.dt)
        e0.record(st)
        for _ in range(reps):
            s.rk_stage(m, pb.dt)
        e1.record(st)
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1) / 1e3 / reps)
    ex = 0.0
    if pb.conns or getattr(pb, "bcs", None):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            s.exchange_ghosts(0)
        e1.record(st)
        torch.cuda.synchronize()
        ex = e0.elapsed_time(e1) / 1e3 / reps
    return out, ex


def roofline(pb, precision, stage_times, ex_time, curvilinear, pk, peak_kind, traffic, rates):
    """Roofline of the fused stage kernel: algorithmic work per launch over
    the launch's average CUDA-event time (the ghost fill subtracted).  The
    FP64-accurate forms are bound by arithmetic: algorithmic FP64 operations
    (the oracle's counts) against the measured peak of their arithmetic; the
    binary32-flux form by HBM: algorithmic bytes against the measured copy
    bandwidth.  The HBM fraction is reported for every form."""
    M = len(stage_times)
    kt = [max(t - ex_time, 1e-12) for t in stage_times]
    byts = [algorithmic_bytes(pb, m + 1, curvilinear, precision) for m in range(M)]
    gbs = sum(byts) / sum(kt) / 1e9
    hbm = pk.get("hbm_gbs", FALLBACK_PEAKS["hbm_gbs"])
    r = {"kernel": "fv_stage_kernel<%s>" % precision, "bytes_per_launch": sum(byts) / M,
         "avg_launch_s": sum(kt) / M}
    r["hbm"] = {"achieved_gbs": gbs, "peak_gbs": hbm, "frac": gbs / hbm, "peak_source": peak_kind}
    if precision == "fp32flux":
        r.update({"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                  "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs, burst copy)"})
    else:
        ops = alu_ops_per_cell(pb.dim, bool(pb.params.get("visc", 0))) * pb.ncells
        achieved = ops / (sum(kt) / M) / 1e9
        peak, how = alu_peak(precision, rates)
        r.update({"bound": "alu", "achieved": achieved, "peak": peak / 1e9, "unit": "G FP64-op/s",
                  "frac": achieved / (peak / 1e9), "ops_per_launch": ops, "peak_source": how,
                  "nominal_peak": nominal_alu_peak(precision) / 1e9})
    # measured DRAM bytes of one launch, for the workload they were captured on
    r["traffic"] = traffic_of(traffic, pb.name, precision)
    return r


def traffic_of(traffic, workload, precision):
    """DRAM bytes per stage launch captured for this workload and form (the
    headline workload at the top level of the summary, others under
    "workloads"), else None."""
    if traffic.get("workload") == workload:
        return traffic.get(precision)
    return traffic.get("workloads", {}).get(workload, {}).get(precision)


def max_over_ranks(x: float, dist, device: str) -> float:
    """The slowest rank's time: replicas run independently, the job ends
    when the last one does."""
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload_config(pb, args, world):
    """The JSON line's config: the workload as both arms name it."""
    curv = pb.blocks[0].nodes is not None
    return {"workload": pb.name, "cells": pb.ncells, "blocks": len(pb.blocks), "rk_stages": len(pb.params["alpha"]),
            "precision": args.precision, "parallelism": "replicas" if world > 1 else "single",
            "l2_flush": "inputs larger than L2 (state+metrics %.0f MB)" % (
                (3 * 5 * 8 * pb.ncells + (80 if curv else 0) * pb.ncells) / 1e6)}


def sig(x, n=4):
    """Round for the compact headline line (floats to n significant digits)."""
    if isinstance(x, float):
        return float("%.*g" % (n, x)) if math.isfinite(x) else None
    if isinstance(x, dict):
        return {k: sig(v, n) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [sig(v, n) for v in x]
    return x


def compact_roofline(r):
    keys = ("bound", "achieved", "peak", "unit", "frac", "traffic", "peak_source")
    out = {k: r[k] for k in keys if k in r}
    out["hbm_frac"] = r["hbm"]["frac"]
    out["kernel"] = r["kernel"]
    out["avg_launch_ms"] = r["avg_launch_s"] * 1e3
    return out


def field_errors(a, b):
    """Per variable max|a - b| / max|b| over a [5][n] field pair (plain
    relative L-infinity, the paper's parallel-vs-serial measure)."""
    a = a.reshape(5, -1)
    b = b.reshape(5, -1)
    out = []
    for v in range(5):
        m = float(np.abs(b[v]).max())
        out.append(float(np.abs(a[v] - b[v]).max()) / m if m > 0 else 0.0)
    return out


def form_errors(pb, stages=100):
    """Each form's error against the binary64 path on the benchmark block:
    one residual of the initial state (plain relative L-infinity per
    variable) and the interior state after `stages` RK stages (the drift).
    The binary64 path itself matches the CPU oracle within 1e-12 (one
    residual) and 1e-10 (100 stages) in the GPU parity tests."""
    import torch
    ref_r = ref_q = None
    out = {}
    b = pb.blocks[0]
    g = (b.nk + 4, b.nj + 4, b.ni + 4)
    for prec in ("fp64", "df64", "fp32flux"):
        s = make_solver(pb, prec, tune=False)
        r = s.residual(0).cpu().numpy()
        for _ in range(stages // s.n_stages):
            s.rk_step(pb.dt, use_graph=True)
        q = s.get_state(0).view(5, *g)[:, 2:-2, 2:-2, 2:-2].reshape(5, -1).cpu().numpy()
        s.close()
        torch.cuda.synchronize()
        if prec == "fp64":
            ref_r, ref_q = r, q
            continue
        out[prec] = {"residual_rel_linf": field_errors(r, ref_r), "drift_stages": stages,
                     "state_rel_linf": field_errors(q, ref_q)}
    return out


def run_gpu(args):
    import torch
    import paper_2012_02925_gb300 as fv
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    rates = fv.probe_alu_rates()
    pb = workload(args.workload)
    curv = pb.blocks[0].nodes is not None
    s = make_solver(pb, args.precision, args.tile, args.kchunk)
    M = s.n_stages
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(args.warmup):
            s.rk_step(pb.dt, use_graph=True)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        step_ms = []
        elapsed = time_steps(s, pb, args.steps, 0, per_step=step_ms)
    if dist:
        elapsed = max_over_ranks(elapsed, dist, "cuda")
    cell_updates = pb.ncells * M * args.steps * world
    value = cell_updates / elapsed / 1e9
    pk, peak_kind = peaks()
    traffic = load_traffic()
    stage_times, ex_time = time_stage_kernels(s, pb, min(20, max(3, args.steps // 2)))
    roof = roofline(pb, args.precision, stage_times, ex_time, curv, pk, peak_kind, traffic, rates)
    # end to end through the public API with host buffers
    e2e = run_e2e(s, pb, min(40, max(3, args.steps // 4)), dist, world)
    launch = s.launch()
    s.close()
    if rank == 0:
        print(json.dumps({"headline_launch": launch, "roofline": sig(roof)}))
    launches_per_step = M * (1 + (1 if pb.conns else 0) + (1 if getattr(pb, "bcs", None) else 0))
    forms = []
    if args.variants and rank == 0 and world == 1:
        variants = run_variants(args, pk, peak_kind, traffic, rates)
        for v in variants:
            print(json.dumps({"variant": sig(v)}))
        try:
            adj = run_adjoint(rates=rates, pk=pk, peak_kind=peak_kind)
        except Exception as e:  # report, do not hide
            adj = {"error": str(e)}
        print(json.dumps({"adjoint": sig(adj)}))
        errs = form_errors(pb)
        for v in variants:
            if v.get("workload") == pb.name and v.get("precision") in ("df64", "fp32flux"):
                f = {"form": v["precision"], "value": v["value"], "vs_fp64": v["value"] / value,
                     "bound": v["roofline"]["bound"], "frac": v["roofline"]["frac"],
                     "hbm_frac": v["roofline"]["hbm"]["frac"]}
                e = errs.get(v["precision"], {})
                f["err_residual"] = max(e.get("residual_rel_linf", [float("nan")]))
                f["drift_100_stages"] = sig(e.get("state_rel_linf"), 2)
                forms.append(f)
        for v in variants:
            if v.get("blocks", 1) > 1 and "error" not in v:
                forms.append({"form": "batched %d blocks %s" % (v["blocks"], v["precision"]), "value": v["value"],
                              "vs_fp64": v["value"] / value, "bound": v["roofline"]["bound"],
                              "frac": v["roofline"]["frac"], "hbm_frac": v["roofline"]["hbm"]["frac"]})
    result = {
        "metric": "Gcell-updates/s per RK stage",
        "value": value,
        "unit": "Gcell-updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": elapsed / args.steps * 1e3,
        # the K timed steps as repeats (an event after each): their spread
        "spread": {"repeats": len(step_ms), "min_ms": min(step_ms), "median_ms": statistics.median(step_ms),
                   "max_ms": max(step_ms)},
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp64": "f64", "df64": "f64 state / f32x2 double-float arithmetic",
                  "fp32flux": "f64 state / f32 flux / f32x2+f64 accumulate+update"}[args.precision],
        "data": "synthetic",
        "config": workload_config(pb, args, world),
        "roofline": compact_roofline(roof),
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk.summary(),
        "forms": forms,
    }
    if rank == 0 and world == 1 and not args.no_cpu:
        result["cpu_baseline"] = cpu_baseline(args.workload)
    if rank == 0:
        print(json.dumps(sig(result)))
    if dist:
        dist.destroy_process_group()


def run_e2e(s, pb, steps, dist=None, world=1):
    """Same metric through the public API with HOST buffers: per step the
    state goes host->device (pinned), one RK step runs, and the residual norms
    of the state the step starts from (10 doubles, recorded by the step's
    first stage through the residual monitor) come back to the host.

    Two ways: overlapped (the reported value) - each step's state is uploaded
    on a copy stream into the handle's staging buffer (fv_stage_state) while
    the previous step computes, then set from it on the compute stream
    (fv_set_state_staged); and serial (set_state from the host buffer, step,
    norms, one after the other)."""
    import torch
    host = torch.from_numpy(pb.q).pin_memory()
    s.set_monitor(True)
    comp = torch.cuda.current_stream()

    def serial_step():
        s.set_state(host)
        s.rk_step(pb.dt, use_graph=True)
        s.monitor_norms()

    copy = torch.cuda.Stream()
    uploaded, consumed = torch.cuda.Event(), torch.cuda.Event()
    s.stage_state(host, stream=copy.cuda_stream)
    uploaded.record(copy)

    def overlapped_step():
        comp.wait_event(uploaded)
        s.set_state_staged()
        consumed.record(comp)
        copy.wait_event(consumed)                       # staging buffer free again
        s.stage_state(host, stream=copy.cuda_stream)    # the next step's input ...
        uploaded.record(copy)
        s.rk_step(pb.dt, use_graph=True)                # ... uploads while this one runs
        s.monitor_norms()

    out = {}
    for name, step in (("serial", serial_step), ("overlapped", overlapped_step)):
        step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(steps):
            step()
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        if dist:
            el = max_over_ranks(el, dist, "cuda")
        # whole job: every rank's cells over the slowest rank's time
        out[name] = pb.ncells * s.n_stages * steps * world / el / 1e9
    s.set_monitor(False)
    return {"value": out["overlapped"], "unit": "Gcell-updates/s",
            "h2d_bytes_per_step": int(pb.q.nbytes) * world, "d2h_bytes_per_step": 80 * world,
            "upload": "overlapped (copy stream)", "serial_value": out["serial"]}


def run_adjoint(n=96, nstages=50, rates=None, pk=None, peak_kind=None):
    """Discrete adjoint workload: 96^3 curvilinear block, van Albada, Harten
    fix on every eigenvalue, J = integrated pressure on the k=0 face after 50
    RK stages; forward with stage checkpoints, then the VJP chain.  The face
    sweeps run in binary64 and in double-float arithmetic
    (fv_set_adjoint_arith); the forward binary64 stage of the same block is
    timed beside them."""
    import torch
    import paper_2012_02925_gb300 as fv
    from paper_2012_02925_gb300.autograd import run_stages
    pb = cases.mms_3d(n, curvilinear=True, with_source=False, limiter=2, fix_all=1)
    s = fv.Solver.from_problem(pb, precision="fp64")
    q0 = torch.from_numpy(pb.q).cuda()
    s.set_state(q0)
    b = pb.blocks[0]
    g = (b.nk + 4, b.nj + 4, b.ni + 4)
    st = torch.cuda.current_stream()

    def J(q):
        Q = q.view(5, *g)[:, 2, 2:-2, 2:-2].reshape(5, -1)
        return ((0.4 * (Q[4] - 0.5 * (Q[1] ** 2 + Q[2] ** 2 + Q[3] ** 2) / Q[0]))).sum()

    def timed(fn, reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fn()
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    fwd_s = timed(lambda: s.rk_stage(2, pb.dt), 10)
    out = {"workload": pb.name + "_adjoint", "stages": nstages, "cells": pb.ncells, "unit": "Gcell-updates/s",
           "forward_fp64_stage_ms": fwd_s * 1e3}
    lam = torch.randn(s.field_size, dtype=torch.float64, device="cuda")
    li = torch.empty_like(lam)
    l0 = torch.zeros_like(lam)
    for arith in ("fp64", "df64"):
        s.set_adjoint_arith(arith)
        x = q0.clone().requires_grad_(True)
        J(run_stages(s, x, pb.dt, nstages)).backward()   # warm-up (allocates adjoint scratch)
        torch.cuda.synchronize()
        x = q0.clone().requires_grad_(True)
        t0 = time.perf_counter()
        y = run_stages(s, x, pb.dt, nstages)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        J(y).backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        vjp_s = timed(lambda: s.adjoint_vjp(2, pb.dt, q0, lam, li, l0), 5)
        r = {"forward_with_checkpoints_s": t1 - t0, "backward_s": t2 - t1, "vjp_stage_ms": vjp_s * 1e3,
             "vjp_value": pb.ncells / vjp_s / 1e9, "vjp_over_forward_stage": vjp_s / fwd_s}
        if rates is not None:
            # one VJP stage reads the checkpoint (40 B) and lambda_out (40 B),
            # the metrics (80 B), and writes lambda_in (40 B) and updates
            # lambda_Q0 (80 B): 280 B per cell
            hbm = pk.get("hbm_gbs", FALLBACK_PEAKS["hbm_gbs"])
            r["hbm_frac"] = 280.0 * pb.ncells / vjp_s / 1e9 / hbm
        out[arith] = r
    s.close()
    return out


def run_variants(args, pk, peak_kind, traffic, rates):
    out = []
    specs = [(w, p) for w in args.variant_workloads.split(",") for p in args.variant_precisions.split(",")]
    cache = {}
    for wname, prec in specs:
        if wname == args.workload and prec == args.precision:
            continue
        try:
            if wname not in cache:
                cache.clear()
                cache[wname] = workload(wname)
            pb = cache[wname]
            curv = pb.blocks[0].nodes is not None
            big = pb.ncells > 3e7
            s = make_solver(pb, prec, reps=1 if big else 3)
            steps = 3 if big else min(10, max(3, args.steps // 2))
            el = time_steps(s, pb, steps, 3)
            st, ex = time_stage_kernels(s, pb, 3)
            out.append({"workload": pb.name, "precision": prec, "blocks": len(pb.blocks), "cells": pb.ncells,
                        "value": pb.ncells * s.n_stages * steps / el / 1e9, "unit": "Gcell-updates/s",
                        "launch": s.launch(), "ghost_fill_s": ex,
                        "roofline": roofline(pb, prec, st, ex, curv, pk, peak_kind, traffic, rates)})
            s.close()
        except Exception as e:  # report, do not hide
            out.append({"workload": wname, "precision": prec, "error": str(e)})
    return out


# ---------------------------------------------------------------------------
# CPU oracle arm
# ---------------------------------------------------------------------------

def oracle_sample(name: str):
    """Bounded sample of the workload: for the 128^3 block, its first 16
    k-planes (same nodes, state, ghosts from the neighbouring planes and
    source) - 262,144 cells."""
    pb = workload(name)
    if name != "mms128":
        return pb, "full workload"
    b = pb.blocks[0]
    nk = 16
    q = cases.unpack_state(pb.blocks, pb.q)[0][:, :nk + 4].copy()
    nb = cases.BlockDesc(b.ni, b.nj, nk, b.nodes[:nk + 1].copy())
    src = [pb.source[0][:, :nk].copy()]
    sp = cases.Problem([nb], [], 3, cases.pack_state([nb], [q]), src, pb.dt, dict(pb.params), pb.name + "_k16")
    return sp, "first 16 of 128 k-planes of the 128^3 block (262,144 cells), full RK steps"


def cpu_baseline(name: str, min_seconds: float = 10.0, max_steps: int = 400):
    """The oracle as it stands on the host cores: whole RK steps on the
    bounded sample, repeated until at least ``min_seconds`` have elapsed."""
    import oracle
    cores = len(os.sched_getaffinity(0))
    sp, desc = oracle_sample(name)
    o = oracle.Oracle(sp, threads=cores)
    q = sp.q.copy()
    M = len(sp.params["alpha"])
    q = o.run(q, sp.dt, M)          # warm-up step (thread pool, page faults)
    steps = 0
    t0 = time.perf_counter()
    while steps < max_steps and (time.perf_counter() - t0) < min_seconds:
        q = o.run(q, sp.dt, M)
        steps += 1
    el = time.perf_counter() - t0
    # the same on one core (the paper compares its GPU codes with 1 and 16
    # CPU cores): whole RK steps for at least 3 s
    o1 = oracle.Oracle(sp, threads=1)
    q1 = sp.q.copy()
    steps1 = 0
    t1 = time.perf_counter()
    while steps1 < max_steps and (time.perf_counter() - t1) < 3.0:
        q1 = o1.run(q1, sp.dt, M)
        steps1 += 1
    el1 = time.perf_counter() - t1
    return {"value": sp.ncells * M * steps / el / 1e9, "unit": "Gcell-updates/s", "cores": cores,
            "kind": "oracle", "sample": desc + ", %d step(s) of %d stages after one warm-up step, %.1f s" % (steps, M, el),
            "single_core": {"value": sp.ncells * M * steps1 / el1 / 1e9, "cores": 1,
                            "sample": "the same sample, %d step(s), %.1f s" % (steps1, el1)}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    cores = len(os.sched_getaffinity(0))
    sp, desc = oracle_sample(args.workload)
    o = oracle.Oracle(sp, threads=cores)
    M = len(sp.params["alpha"])
    q = sp.q.copy()
    for _ in range(args.warmup):
        q = o.run(q, sp.dt, M)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        q = o.run(q, sp.dt, M)
    el = time.perf_counter() - t0
    v = sp.ncells * M * args.steps / el / 1e9
    res = {"impl": "reference", "metric": "Gcell-updates/s per RK stage", "value": v, "unit": "Gcell-updates/s",
           "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": workload_config(workload(args.workload), args, int(os.environ.get("WORLD_SIZE", "1"))),
           "cpu_baseline": {"value": v, "unit": "Gcell-updates/s", "cores": cores, "kind": "oracle",
                            "sample": desc + " (the oracle computes in binary64), %d timed step(s) of %d stages"
                            % (args.steps, M)},
           "e2e": {"value": v, "unit": "Gcell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(res))


def run_peaks():
    """Measured arithmetic rates of the current GPU (fv_probe_alu_rates) and
    the peaks the forms are graded against, one JSON line."""
    import torch
    import paper_2012_02925_gb300 as fv
    torch.cuda.set_device(0)
    rates = fv.probe_alu_rates()
    out = {"gpu": torch.cuda.get_device_name(0), "rates_per_s": rates,
           "peaks": {p: dict(zip(("value_per_s", "how"), alu_peak(p, rates))) for p in ("fp64", "df64")},
           "nominal": {p: nominal_alu_peak(p) for p in ("fp64", "df64")}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # 200 steps of the 128^3 block: a timed region of a few seconds, long
    # enough for many clock samples
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="fvgb", choices=["fvgb", "reference"])
    ap.add_argument("--workload", default="mms128")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "df64", "fp32flux"])
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--kchunk", type=int, default=0)
    ap.add_argument("--variants", type=int, default=1)
    ap.add_argument("--variant-workloads",
                    default="vortex,mms128,multiblock,large,mms128+vl,mms128+sw,inlet,ogrid,mms128+ns,ogrid+ns")
    ap.add_argument("--variant-precisions", default="fp64,df64,fp32flux")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--peaks", action="store_true")
    ap.add_argument("--adjoint", action="store_true", help="the adjoint workload's line only")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.peaks:
        run_peaks()
    elif args.adjoint:
        import torch
        import paper_2012_02925_gb300 as fv
        torch.cuda.set_device(0)
        pk, kind = peaks()
        print(json.dumps({"adjoint": sig(run_adjoint(rates=fv.probe_alu_rates(), pk=pk, peak_kind=kind))}))
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
