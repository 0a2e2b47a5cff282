#!/usr/bin/env python3
"""Benchmark of the lattice-QCD fermion solve hot path on one GB300 (or N replicas).

Workload (the paper's 32^3 x 64 Wilson lattice, Sec. V): Wilson fermion on
32^3 x 64, smoothed-random SU(3) links (eps = 0.2, seed 2), kappa = 0.125,
periodic space / antiperiodic time, complex Z2 noise source (seed 0); the
FP32/FP16 link copies use 12-real reconstruction.

One step = one pass of the hot path on that input:
  1. the standalone even-odd hopping stencil D_eo in FP32 (NDSLASH launches)
     and in FP64 (one launch), on internal-layout device buffers;
  2. the mixed-precision even-odd BiCGStab solve (FP32 inner iterations,
     IEEE-FP64 reliable updates: true residual, solution accumulation and
     reductions in FP64) to |b - M x| / |b| <= 1e-10 on the full system,
     from canonical device buffers (source preparation, solve, reconstruction
     and the final FP64 true residual included).
`value` is the whole-step dslash rate: 1320 flop per output site for every
half-dslash the step executes (standalone ones and those inside the solve),
divided by the step's device time.  The plain FP64 GPU solve of the same
system is timed once after the timed steps and reported beside the mixed one.

--impl reference times the FP64 CPU oracle on the same workload (a bounded
sample: the hopping term on the full lattice) on this machine's host cores.
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
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
from paper_1712_01505_gb300 import metrics  # noqa: E402  (flop / byte model, no GPU code)

METRIC = "dslash GFLOP/s & %HBM roofline; mixed vs FP64 solve time to rel. residual 1e-10"
L = (32, 32, 32, 64)
BC = (1, 1, 1, -1)
EPS, GAUGE_SEED, KAPPA, SRC_SEED = 0.2, 2, 0.125, 0
RECON = 12
TOL = 1e-10
# reliable-update factor of the FP16-inner solve, measured fastest for it on this system: 0.01 and
# 5e-3 take five outer steps, 3e-3 to 3e-4 four (the FP32-inner solve: 1e-5, two)
DELTA16 = 2e-3
NDSLASH = 10
FLOP_SITE = metrics.HOP_FLOP_SITE      # 1320 per output site of one half-dslash (hopping term)
BYTES_SITE_FP32 = {r: int(metrics.hop_compulsory_bytes("f32", r)) for r in (12, 18)}  # links + in + out
BYTES_SITE_FP64 = int(metrics.hop_compulsory_bytes("f64", 18))
BYTES_SITE_FP16 = int(metrics.hop_compulsory_bytes("f16", RECON))
WORKLOAD = "wilson_32x32x32x64_kappa0.125_eps0.2_z2"
PROFILE = os.path.join(ROOT, "profiles", "wilson_dslash_fp32_32x32x32x64.md")
KERNEL_SOURCES = ["paper_1712_01505_gb300/csrc/wilson.cu", "paper_1712_01505_gb300/csrc/stencil.cuh",
                  "paper_1712_01505_gb300/csrc/common.cuh"]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"




def kernel_hash():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """dram bytes per launch of the FP32 D_eo from the committed ncu summary, if the kernel is unchanged."""
    if not os.path.exists(PROFILE):
        return None
    txt = open(PROFILE).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    hsh = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", txt)
    if not m or not hsh or hsh.group(1) != kernel_hash():
        return None
    return float(m.group(1))


class Clocks:
    """nvidia-smi sampling (200 ms) during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(U, psi, budget_s=12.0, solve=True):
    """The FP64 oracle's hopping term D_eo on the full lattice, timed on the host cores (all of
    them and one), and its FP64 solve of the benchmark system."""
    from oracle import oracle as ora

    par = ora.parity(L)
    inp = psi.copy()
    inp[par == 0] = 0
    ora.hop(L, BC, U, inp, out_parity=0)  # warm-up (page-in, thread pool)
    reps, t0 = 0, time.perf_counter()
    while True:
        ora.hop(L, BC, U, inp, out_parity=0)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or reps >= 50:
            break
    Vh = int(np.prod(L)) // 2
    gflops = FLOP_SITE * Vh * reps / el / 1e9
    cores = ora.num_threads()
    # the same on one thread, a shorter sample
    ora.set_num_threads(1)
    try:
        reps1, t0 = 0, time.perf_counter()
        while True:
            ora.hop(L, BC, U, inp, out_parity=0)
            reps1 += 1
            el1 = time.perf_counter() - t0
            if el1 >= budget_s / 4 or reps1 >= 10:
                break
    finally:
        ora.set_num_threads(cores)
    out = {"value": round(gflops, 4), "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
           "sample": f"{reps} oracle FP64 D_eo applications on the full 32^3x64 lattice "
                     f"({Vh} output sites each, {el:.1f} s)",
           "value_1thread": round(FLOP_SITE * Vh * reps1 / el1 / 1e9, 4),
           "sample_1thread": f"{reps1} applications on one thread ({el1:.1f} s)"}
    if solve:  # the oracle's FP64 even-odd BiCGStab on the same system, to the same 1e-10
        t0 = time.perf_counter()
        _, it, res = ora.wilson_solve(L, BC, KAPPA, U, psi, tol=TOL)
        out["solve_s"] = round(time.perf_counter() - t0, 2)
        out["solve_iters"] = it
        out["solve_true_resid"] = res
    return out


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1712_01505_gb300 import inputs
    from oracle import oracle as ora

    U = inputs.gauge_field(L, EPS, GAUGE_SEED)
    psi = inputs.z2_source((int(np.prod(L)), 4, 3), SRC_SEED)
    par = ora.parity(L)
    inp = psi.copy()
    inp[par == 0] = 0
    Vh = int(np.prod(L)) // 2
    for _ in range(args.warmup):
        ora.hop(L, BC, U, inp, out_parity=0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ora.hop(L, BC, U, inp, out_parity=0)
    el = time.perf_counter() - t0
    val = FLOP_SITE * Vh * args.steps / el / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(val, 4), "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "lattice": list(L), "kappa": KAPPA,
                                              "eps": EPS, "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": round(val, 4), "unit": "GFLOP/s", "cores": ora.num_threads(),
                             "kind": "oracle",
                             "sample": f"each step: one FP64 oracle D_eo on the full lattice ({Vh} sites)"},
            "e2e": {"value": round(val, 4), "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-solve", action="store_true")
    ap.add_argument("--profile", default="none", choices=["none", "dslash", "step", "mhat", "cg"],
                    help="for ncu: 'dslash' runs only the standalone FP32 D_eo launches, 'step' one step "
                         "between cudaProfilerStart/Stop (use ncu --profile-from-start off); no JSON line")
    ap.add_argument("--profile-prec", default="f32", choices=["f32", "f64", "df64", "f16"],
                    help="precision of the D_eo launches of --profile dslash (and of the domain-wall hop / "
                         "Mhat of --workload dwf --profile dslash / mhat); f16 with --profile step: the "
                         "step's solve runs FP16 inner iterations")
    ap.add_argument("--workload", default="wilson32", choices=["wilson32", "dwf", "batched", "force", "dd"],
                    help="wilson32 (default, the bench line); the others characterise the other "
                         "configurations (domain-wall CG, 12-rhs propagator, force) and print their own line")
    ap.add_argument("--outer", default="f64", choices=["f64", "df64"],
                    help="precision of the outer steps of the mixed solve: f64 = IEEE FP64 stencil (the "
                         "default), df64 = double-float stencil (FP32 pairs); the final residual is IEEE FP64 "
                         "either way")
    ap.add_argument("--delta", type=float, default=None,
                    help="reliable-update factor of the mixed solves (default: 1e-5 for the FP32 Wilson solves "
                         "of the bench line and the batched workload, the library's per-precision default "
                         "for domain-wall)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "wilson32":
        from bench_configs import run_workload

        return run_workload(args)

    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1712_01505_gb300 import inputs, qcd
    from paper_1712_01505_gb300.replicas import replica_reduce

    V = int(np.prod(L))
    Vh = V // 2
    U = inputs.gauge_field(L, EPS, GAUGE_SEED)
    psi = inputs.z2_source((V, 4, 3), SRC_SEED)
    g = qcd.Gauge.load(torch.from_numpy(U).to(dev), L, BC, recon=RECON)
    f = qcd.wilson(KAPPA)
    stream = torch.cuda.current_stream(dev)
    b_dev = torch.from_numpy(psi).to(dev)
    x_dev = torch.zeros_like(b_dev)
    # internal-layout buffers for the standalone stencil
    nb32 = qcd.field_bytes(g, f, "f32")
    nb64 = qcd.field_bytes(g, f, "f64")
    in32 = torch.empty(nb32, dtype=torch.uint8, device=dev)
    out32 = torch.empty(nb32, dtype=torch.uint8, device=dev)
    in64 = torch.empty(nb64, dtype=torch.uint8, device=dev)
    out64 = torch.empty(nb64, dtype=torch.uint8, device=dev)
    qcd.field_pack(g, f, "f32", 1, b_dev, in32)
    qcd.field_pack(g, f, "f64", 1, b_dev, in64)
    delta = 1e-5 if args.delta is None else args.delta
    solve_kw = dict(method=qcd.BICGSTAB, tol=TOL, inner="f32", use_graph=True, graph_chunk=32, delta=delta,
                    outer=args.outer)
    if args.profile == "step" and args.profile_prec == "f16":  # the FP16-inner solve of the f16_inner line
        solve_kw = dict(solve_kw, inner="f16", delta=DELTA16)

    ev_d0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_d1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_s0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_s1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]

    def step(i=None):
        if i is not None:
            ev_d0[i].record(stream)
        for _ in range(NDSLASH):
            qcd.dslash(g, f, "D_EO", in32, out32, prec="f32", layout=qcd.INTERNAL)
        if i is not None:
            ev_d1[i].record(stream)
        qcd.dslash(g, f, "D_EO", in64, out64, prec="f64", layout=qcd.INTERNAL)
        if i is not None:
            ev_s0[i].record(stream)
        x_dev.zero_()
        info, _ = qcd.solve(g, f, b_dev, x_dev, **solve_kw)
        if i is not None:
            ev_s1[i].record(stream)
        return info[0]

    if args.profile == "dslash":
        pp = args.profile_prec
        if pp == "f32":
            pin, pout = in32, out32
        elif pp == "f64":
            pin, pout = in64, out64
        else:
            pin = torch.empty(qcd.field_bytes(g, f, pp), dtype=torch.uint8, device=dev)
            pout = torch.empty_like(pin)
            qcd.field_pack(g, f, pp, 1, b_dev, pin)
        for _ in range(3):  # tuning and warm-up, then the profiled launches
            qcd.dslash(g, f, "D_EO", pin, pout, prec=pp, layout=qcd.INTERNAL)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        for _ in range(NDSLASH if pp == "f32" else 3):
            qcd.dslash(g, f, "D_EO", pin, pout, prec=pp, layout=qcd.INTERNAL)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print("profile dslash done", flush=True)
        return
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if args.profile == "step":
        torch.cuda.profiler.start()
        info = step()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(f"profile step done: {info}", flush=True)
        return
    if dist:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    n0 = qcd.kernel_launches()
    torch.cuda.synchronize()
    t_start.record(stream)
    infos = [step(i) for i in range(args.steps)]
    t_end.record(stream)
    torch.cuda.synchronize()
    n_launch = qcd.kernel_launches() - n0
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    d_ms = [ev_d0[i].elapsed_time(ev_d1[i]) / NDSLASH for i in range(args.steps)]
    s_ms = [ev_s0[i].elapsed_time(ev_s1[i]) for i in range(args.steps)]
    dslash_avg_ms = sum(d_ms) / len(d_ms)
    for inf in infos:
        if not inf["converged"] or inf["true_resid"] > TOL:
            raise SystemExit(f"solve failed to converge: {inf}")

    def hops_in_solve(inf, outer=args.outer):
        # 4 inner half-dslashes per BiCGStab iteration, 1 for the source and 2 per outer step
        # (none before the first since x0 = 0).  IEEE-FP64 outer steps reconstruct x_o and form
        # the full-system residual themselves, so the last one ends the solve; double-float
        # outer steps add the reconstruction and the even half of the final FP64 residual.
        return 4 * inf["iters"] + 1 + 2 * inf["outer_updates"] + (2 if outer == "df64" else 0)

    hops = sum(NDSLASH + 1 + hops_in_solve(inf) for inf in infos)
    # whole job: the slowest rank's time, every rank's work
    total_ms, hops_all = replica_reduce(total_ms, hops, dist, dev)
    flops = FLOP_SITE * Vh * hops_all
    value = flops / (total_ms / 1e3) / 1e9
    hbm, peak_kind = peaks()
    alg_bytes = BYTES_SITE_FP32[RECON] * Vh
    achieved = alg_bytes / (dslash_avg_ms / 1e3) / 1e9
    traffic = profiled_traffic()

    # ---- plain FP64 GPU solve (the comparison), once
    fp64 = None
    if not args.no_fp64_solve:
        kw64 = dict(method=qcd.BICGSTAB, tol=TOL, inner="f64", use_graph=True, graph_chunk=32)
        x_dev.zero_()
        qcd.solve(g, f, b_dev, x_dev, **kw64)  # warm-up: stencil tuning, workspace, graphs
        x_dev.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info64, _ = qcd.solve(g, f, b_dev, x_dev, **kw64)
        e1.record(stream)
        torch.cuda.synchronize()
        fp64 = {"ms": round(e0.elapsed_time(e1), 3), "iters": info64[0]["iters"],
                "true_resid": info64[0]["true_resid"]}

    # ---- the same mixed solve with the other outer precision, once (for comparison)
    other = "f64" if args.outer == "df64" else "df64"
    x_dev.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    qcd.solve(g, f, b_dev, x_dev, **dict(solve_kw, outer=other))  # warm-up (workspace, graphs)
    x_dev.zero_()
    e0.record(stream)
    info_o, _ = qcd.solve(g, f, b_dev, x_dev, **dict(solve_kw, outer=other))
    e1.record(stream)
    torch.cuda.synchronize()
    other_outer = {"outer": other, "ms": round(e0.elapsed_time(e1), 3), "iters": info_o[0]["iters"],
                   "updates": info_o[0]["outer_updates"], "true_resid": info_o[0]["true_resid"]}

    # ---- the mixed solve with FP16 inner iterations (per-site scaled spinors, 12-real FP16
    # links, FP32 arithmetic), once, and the standalone FP16 D_eo
    x_dev.zero_()
    kw16 = dict(solve_kw, inner="f16", delta=DELTA16)
    qcd.solve(g, f, b_dev, x_dev, **kw16)  # warm-up (tuning, workspace, graphs)
    x_dev.zero_()
    e0.record(stream)
    info16, _ = qcd.solve(g, f, b_dev, x_dev, check=False, **kw16)
    e1.record(stream)
    torch.cuda.synchronize()
    f16_inner = {"ms": round(e0.elapsed_time(e1), 3), "delta": DELTA16, "iters": info16[0]["iters"],
                 "updates": info16[0]["outer_updates"], "true_resid": info16[0]["true_resid"],
                 "converged": bool(info16[0]["converged"])}
    nb16 = qcd.field_bytes(g, f, "f16")
    in16 = torch.empty(nb16, dtype=torch.uint8, device=dev)
    out16 = torch.empty(nb16, dtype=torch.uint8, device=dev)
    qcd.field_pack(g, f, "f16", 1, b_dev, in16)
    for _ in range(3):
        qcd.dslash(g, f, "D_EO", in16, out16, prec="f16", layout=qcd.INTERNAL)
    e0.record(stream)
    for _ in range(10):
        qcd.dslash(g, f, "D_EO", in16, out16, prec="f16", layout=qcd.INTERNAL)
    e1.record(stream)
    torch.cuda.synchronize()
    d16_ms = e0.elapsed_time(e1) / 10
    del in16, out16

    # ---- standalone FP64 D_eo rate (ALU-bound on GB300)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(3):
        qcd.dslash(g, f, "D_EO", in64, out64, prec="f64", layout=qcd.INTERNAL)
    e1.record(stream)
    torch.cuda.synchronize()
    d64_ms = e0.elapsed_time(e1) / 3
    # the FP64 rate of this GPU, measured live (the FP64 stencil's roofline denominator)
    from bench_configs import _fp64_peak_tflops
    fp64_peak = _fp64_peak_tflops()
    # ---- standalone double-float D_eo (the outer-step stencil)
    nbdf = qcd.field_bytes(g, f, "df64")
    indf = torch.empty(nbdf, dtype=torch.uint8, device=dev)
    outdf = torch.empty(nbdf, dtype=torch.uint8, device=dev)
    qcd.field_pack(g, f, "df64", 1, b_dev, indf)
    qcd.dslash(g, f, "D_EO", indf, outdf, prec="df64", layout=qcd.INTERNAL)
    e0.record(stream)
    for _ in range(3):
        qcd.dslash(g, f, "D_EO", indf, outdf, prec="df64", layout=qcd.INTERNAL)
    e1.record(stream)
    torch.cuda.synchronize()
    ddf_ms = e0.elapsed_time(e1) / 3
    del indf, outdf

    # ---- end to end through the C ABI with host buffers (pinned), one step
    b_host = torch.from_numpy(psi).pin_memory().numpy()
    x_host = torch.zeros((V, 4, 3), dtype=torch.complex128).pin_memory().numpy()
    o_host = torch.zeros((V, 4, 3), dtype=torch.complex128).pin_memory().numpy()
    e2e_ms = []
    for rep in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        qcd.dslash(g, f, "D_EO", b_host, o_host, prec="f32")
        info_e, _ = qcd.solve(g, f, b_host, x_host, **solve_kw)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_hops = 1 + hops_in_solve(info_e[0])
    e2e_t, e2e_hops_all = replica_reduce(min(e2e_ms), e2e_hops, dist, dev)
    e2e_val = FLOP_SITE * Vh * e2e_hops_all / (e2e_t / 1e3) / 1e9
    spinor_bytes = V * 12 * 16

    mixed_ms = statistics.median(s_ms)
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic: smoothed-random SU(3) links and Z2 noise source (seeded)",
        "config": {"workload": WORKLOAD, "lattice": list(L), "kappa": KAPPA, "eps": EPS, "recon": RECON,
                   "solver": "EO BiCGStab, FP32 inner + reliable updates in "
                             + ("double-float (FP32 pairs)" if args.outer == "df64" else "IEEE FP64")
                             + " (FP64 solution and reductions), FP64 final residual, CUDA graph chunks of 32",
                   "outer": args.outer,
                   "tol": TOL, "ndslash_per_step": NDSLASH, "delta": delta,
                   "l2": "inputs larger than L2 (links 403 MB, each parity vector 101 MB)",
                   "parallelism": f"replicas{world}" if world > 1 else "single"},
        "roofline": {"bound": "hbm", "kernel": "k_hop<FP32,12-real> (D_eo)", "achieved": round(achieved, 1),
                     "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                     "traffic": traffic, "algorithmic_bytes": alg_bytes,
                     "note": f"peak of {peak_kind} (copy bandwidth); {BYTES_SITE_FP32[RECON]} B per output site"},
        "dslash": {"fp32_ms": round(dslash_avg_ms, 4),
                   "fp32_gflops": round(FLOP_SITE * Vh / (dslash_avg_ms / 1e3) / 1e9, 1),
                   "fp64_ms": round(d64_ms, 4),
                   "fp64_gflops": round(FLOP_SITE * Vh / (d64_ms / 1e3) / 1e9, 1),
                   "fp64_bound": "alu", "fp64_peak_tflops": round(fp64_peak, 4),
                   "fp64_peak_note": "cuBLAS DGEMM 4096^3 measured in this run",
                   "fp64_frac": round(FLOP_SITE * Vh / (d64_ms / 1e3) / 1e12 / fp64_peak, 4),
                   "fp64_gbs": round(BYTES_SITE_FP64 * Vh / (d64_ms / 1e3) / 1e9, 1),
                   "df64_ms": round(ddf_ms, 4),
                   "df64_gflops": round(FLOP_SITE * Vh / (ddf_ms / 1e3) / 1e9, 1),
                   "df64_gbs": round(BYTES_SITE_FP64 * Vh / (ddf_ms / 1e3) / 1e9, 1),
                   "fp16_ms": round(d16_ms, 4),
                   "fp16_gflops": round(FLOP_SITE * Vh / (d16_ms / 1e3) / 1e9, 1),
                   "fp16_gbs": round(BYTES_SITE_FP16 * Vh / (d16_ms / 1e3) / 1e9, 1),
                   "fp16_frac": round(BYTES_SITE_FP16 * Vh / (d16_ms / 1e3) / 1e9 / hbm, 4)},
        "solve": {"mixed_ms": round(mixed_ms, 3), "mixed_iters": infos[-1]["iters"],
                  "mixed_updates": infos[-1]["outer_updates"], "mixed_true_resid": infos[-1]["true_resid"],
                  "fp64": fp64, "speedup_vs_fp64": round(fp64["ms"] / mixed_ms, 3) if fp64 else None,
                  "other_outer": other_outer, "f16_inner": f16_inner},
        "e2e": {"value": round(e2e_val, 3), "unit": "GFLOP/s", "ms": round(min(e2e_ms), 3),
                "h2d_bytes_per_step": 2 * spinor_bytes, "d2h_bytes_per_step": 2 * spinor_bytes},
        "gpu_launches": n_launch,
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(U, psi)
    if rank == 0:
        print(json.dumps(out), flush=True)
    g.free()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
