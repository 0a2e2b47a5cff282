"""Measurements of the other workloads of the solve path (invoked as `bench.py --workload ...`).

* dwf:     domain-wall 16^3 x 32 x Ls=16, M5 = 1.8, mf = 0.02, eps = 0.2 (seed 3), Gaussian
           source (seed 0): the fifth-dimension hop in FP32 and FP16, and CG on Mhat^dag Mhat
           with FP16 / FP32 inner iterations + FP64 or double-float outer steps against the
           plain FP64 CG, to 1e-10; the same for the Mobius operator with b5 = 1.5, c5 = 0.5;
           BiCGStab on the domain-wall system; the hop as Ls launches of the 4D hop.
* batched: Wilson 24^3 x 48, kappa = 0.124, eps = 0.2 (seed 4), the 12 spin-colour point
           sources at one random site (seed 0): one 12-rhs solve (shared link loads, graph
           chunks, tuned tiles) against 12 single-rhs solves, FP32 inner + FP64, to 1e-10.
* force:   Wilson 16^4, kappa = 0.12, eps = 0.3 (seed 5), Gaussian phi (seed 0): the backward
           pass of S = phi^dag (M^dag M)^-1 phi (adjoint solve + outer-product kernel).
* dd:      the 32^3 x 64 Wilson system cut into 2, 4 or 16 subdomains of one process (domain
           decomposition on one GPU): Mhat and the mixed BiCGStab against the single-domain ones.
Each prints one JSON line.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np
import torch

from paper_1712_01505_gb300 import inputs, metrics, qcd

BC = (1, 1, 1, -1)


def _events():
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _time_launches(fn, n=20, warm=3):
    for _ in range(warm):
        fn()
    e0, e1 = _events()
    e0.record()
    for _ in range(n):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / n


def _peak():
    import os
    p = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    return float(json.load(open(p))["hbm_gbs"]) if os.path.exists(p) else 6800.0


TRAFFIC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles", "workload_kernels_dram_traffic.md")
TRAFFIC_SOURCES = ["paper_1712_01505_gb300/csrc/wilson.cu", "paper_1712_01505_gb300/csrc/stencil.cuh",
                   "paper_1712_01505_gb300/csrc/common.cuh", "paper_1712_01505_gb300/csrc/force.cu"]


def _traffic(key):
    """DRAM bytes per launch of a workload's kernel from the committed ncu summary, if the kernel
    sources still hash to the value recorded there (else None)."""
    import hashlib
    import re

    if not os.path.exists(TRAFFIC):
        return None
    root = os.path.dirname(os.path.abspath(__file__))
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        h.update(open(os.path.join(root, f), "rb").read())
    txt = open(TRAFFIC).read()
    m = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", txt)
    v = re.search(rf"{key}:\s*([0-9.eE+]+)", txt)
    if not m or not v or m.group(1) != h.hexdigest()[:16]:
        return None
    return float(v.group(1))


def _cpu_rate(fn, units, budget_s=6.0, max_reps=20):
    """The oracle `fn` timed on the host cores over a bounded sample: (units per second, reps, seconds)."""
    fn()  # warm-up (page-in, thread pool)
    reps, t0 = 0, time.perf_counter()
    while True:
        fn()
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or reps >= max_reps:
            return units * reps / el, reps, el


def _fp64_peak_tflops():
    """FP64 throughput of this GPU measured live: cuBLAS DGEMM 4096^3 (best of 5 after a warm-up)."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = 0.0
    for _ in range(5):
        e0, e1 = _events()
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, 2.0 * n ** 3 / (e0.elapsed_time(e1) / 1e3) / 1e12)
    return best


def run_dwf(args):
    L, Ls, M5, mf = (16, 16, 16, 32), 16, 1.8, 0.02
    V = int(np.prod(L))
    Vh = V // 2
    U = inputs.gauge_field(L, 0.2, 3)
    b = inputs.gaussian_source((Ls, V, 4, 3), 0)
    dev = torch.device("cuda", 0)
    g = qcd.Gauge.load(torch.from_numpy(U).to(dev), L, BC, recon=12)
    f = qcd.dwf(Ls, M5, mf)
    bd = torch.from_numpy(b).to(dev)
    hop = {}
    for prec, site_b, link_b in (("f32", 96, 48), ("f16", 52, 24)):
        if args.profile in ("dslash", "mhat") and prec != args.profile_prec:
            continue
        nb = qcd.field_bytes(g, f, prec)
        a_ = torch.empty(nb, dtype=torch.uint8, device=dev)
        o_ = torch.empty(nb, dtype=torch.uint8, device=dev)
        qcd.field_pack(g, f, prec, 1, bd, a_)
        if args.profile == "cg":  # ncu: one warmed-up CG solve (inner precision --profile-prec, FP32 or
            # FP16, at the reliable-update factor of the measured solve; IEEE-FP64 outer steps)
            pin = "f16" if args.profile_prec == "f16" else "f32"
            kw = dict(method=qcd.CG_NORMAL, tol=1e-10, inner=pin, use_graph=True, graph_chunk=32,
                      delta=(args.delta or (1e-4 if pin == "f32" else 0.0)), outer=args.outer)
            x = torch.zeros_like(bd)
            qcd.solve(g, f, bd, x, **kw)
            x.zero_()
            torch.cuda.synchronize()
            torch.cuda.profiler.start()
            info, _ = qcd.solve(g, f, bd, x, **kw)
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
            print(f"profile dwf cg done: {info[0]}", flush=True)
            return
        if args.profile != "none":  # ncu: tune, then profile 3 launches of the FP32 hop (or of Mhat)
            op = "MHAT" if args.profile == "mhat" else "D_EO"
            if op == "MHAT":
                qcd.field_pack(g, f, prec, 0, bd, a_)
            for _ in range(3):
                qcd.dslash(g, f, op, a_, o_, prec=prec, layout=qcd.INTERNAL)
            torch.cuda.synchronize()
            torch.cuda.profiler.start()
            for _ in range(3):
                qcd.dslash(g, f, op, a_, o_, prec=prec, layout=qcd.INTERNAL)
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
            print(f"profile dwf {op} done", flush=True)
            return
        ms = _time_launches(lambda: qcd.dslash(g, f, "D_EO", a_, o_, prec=prec, layout=qcd.INTERNAL))
        ms_m = _time_launches(lambda: qcd.dslash(g, f, "MHAT", a_, o_, prec=prec, layout=qcd.INTERNAL), n=10)
        alg = Vh * (8 * link_b + Ls * 2 * site_b)
        hop[prec] = {"hop_ms": round(ms, 4), "hop_gflops": round(metrics.HOP_FLOP_SITE * Vh * Ls / ms / 1e6, 1),
                     "hop_gbs": round(alg / ms / 1e6, 1), "hop_frac": round(alg / ms / 1e6 / _peak(), 4),
                     "mhat_ms": round(ms_m, 4)}
    # repeated-4D comparison (Sec. II B 2, the first option): the fifth-dimension hop as Ls launches
    # of the 4D Wilson hop, each on one slice (links re-read per slice) against one launch over
    # all slices (links loaded once per site for every slice)
    fw = qcd.wilson(0.125)
    nb1 = qcd.field_bytes(g, fw, "f32")
    a1 = [torch.empty(nb1, dtype=torch.uint8, device=dev) for _ in range(Ls)]
    o1 = [torch.empty(nb1, dtype=torch.uint8, device=dev) for _ in range(Ls)]
    for s_ in range(Ls):
        qcd.field_pack(g, fw, "f32", 1, bd[s_], a1[s_])

    def rep4d():
        for s_ in range(Ls):
            qcd.dslash(g, fw, "D_EO", a1[s_], o1[s_], prec="f32", layout=qcd.INTERNAL)

    hop["f32"]["repeated_4d_ms"] = round(_time_launches(rep4d, n=10), 4)
    hop["f32"]["fused_5d_speedup"] = round(hop["f32"]["repeated_4d_ms"] / hop["f32"]["hop_ms"], 3)
    del a1, o1
    res = {}
    # inner precision / outer precision of the mixed solves; "f64" is the plain FP64 CG.  The
    # reliable-update factor is the one measured fastest per inner precision (FP32: 1e-4, three
    # outer steps; FP16: the library's 0.01) unless --delta is given
    for name, inner, outer in (("f16", "f16", "f64"), ("f32", "f32", "f64"), ("f16_df", "f16", "df64"),
                               ("f32_df", "f32", "df64"), ("f64", "f64", "f64")):
        kw = dict(method=qcd.CG_NORMAL, tol=1e-10, inner=inner, use_graph=True, graph_chunk=32,
                  delta=(args.delta or (1e-4 if inner == "f32" else 0.0)), outer=outer)
        x = torch.zeros_like(bd)
        qcd.solve(g, f, bd, x, **kw)  # warm-up (tuning, workspace)
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info, _ = qcd.solve(g, f, bd, x, **kw)
        torch.cuda.synchronize()
        res[name] = {"ms": round((time.perf_counter() - t0) * 1e3, 2), "iters": info[0]["iters"],
                     "updates": info[0]["outer_updates"], "true_resid": info[0]["true_resid"]}
    # BiCGStab on the same system (Sec. II C: the paper's reason for CG here), capped at 4x CG's
    # iteration count
    kw = dict(method=qcd.BICGSTAB, tol=1e-10, inner="f32", use_graph=True, graph_chunk=32, outer="df64",
              maxiter=4 * res["f32_df"]["iters"])
    x = torch.zeros_like(bd)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info, st = qcd.solve(g, f, bd, x, check=False, **kw)
    torch.cuda.synchronize()
    bicg = {"ms": round((time.perf_counter() - t0) * 1e3, 2), "iters": info[0]["iters"],
            "maxiter": kw["maxiter"], "converged": bool(info[0]["converged"]),
            "status": qcd.STATUS_NAMES[st], "true_resid": info[0]["true_resid"]}
    # Mobius (b5 = 1.5, c5 = 0.5: the Shamir kernel scaled by b5 + c5 = 2) on the same lattice
    fm = qcd.mobius(Ls, M5, mf, 1.5, 0.5)
    nb = qcd.field_bytes(g, fm, "f32")
    a_ = torch.empty(nb, dtype=torch.uint8, device=dev)
    o_ = torch.empty(nb, dtype=torch.uint8, device=dev)
    qcd.field_pack(g, fm, "f32", 0, bd, a_)
    mob = {"mhat_ms_f32": round(_time_launches(lambda: qcd.dslash(g, fm, "MHAT", a_, o_, prec="f32",
                                                                  layout=qcd.INTERNAL), n=10), 4)}
    for name, inner, outer in (("f32_df", "f32", "df64"), ("f64", "f64", "f64")):
        kw = dict(method=qcd.CG_NORMAL, tol=1e-10, inner=inner, use_graph=True, graph_chunk=32,
                  delta=(args.delta or 0.0), outer=outer)
        x = torch.zeros_like(bd)
        qcd.solve(g, fm, bd, x, **kw)  # warm-up (tuning, workspace)
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info, _ = qcd.solve(g, fm, bd, x, **kw)
        torch.cuda.synchronize()
        mob[name] = {"ms": round((time.perf_counter() - t0) * 1e3, 2), "iters": info[0]["iters"],
                     "updates": info[0]["outer_updates"], "true_resid": info[0]["true_resid"]}
    mob["speedup_f32_df_vs_f64"] = round(mob["f64"]["ms"] / mob["f32_df"]["ms"], 3)
    # roofline of the dominant kernels: the FP32 hop and the fused hop + W of Mhat (12-real links
    # once per site, Ls spinors in and out; Mhat's second launch also reads x)
    peak = _peak()
    mhat_bytes = 2 * Vh * (8 * 48 + Ls * 2 * 96) + Vh * Ls * 96
    roof = {"bound": "hbm", "kernel": "multi-slice hop, FP32 12-real (k_hop_smp)",
            "achieved": hop["f32"]["hop_gbs"], "peak": peak, "unit": "GB/s", "frac": hop["f32"]["hop_frac"],
            "algorithmic_bytes": Vh * (8 * 48 + Ls * 2 * 96), "traffic": _traffic("dwf_hop_f32"),
            "note": "peak of measured copy bandwidth; 8 x 48 B links per 4D site + 96 B in + 96 B out per "
                    "(site, slice)",
            "mhat_fused_f32": {"bytes": mhat_bytes, "ms": hop["f32"]["mhat_ms"],
                               "frac": round(mhat_bytes / hop["f32"]["mhat_ms"] / 1e6 / peak, 4)}}
    cpu = None
    if not getattr(args, "no_cpu_baseline", False):
        from oracle import oracle as ora

        par = ora.parity(L)
        src = b.copy()
        src[:, par == 0] = 0
        rate, reps, el = _cpu_rate(lambda: ora._hop5(L, BC, U, src, out_parity=0), metrics.HOP_FLOP_SITE * Vh * Ls)
        rate_d, reps_d, el_d = _cpu_rate(lambda: ora.dw(L, BC, Ls, M5, mf, U, b), 1.0)
        cpu = {"value": round(rate / 1e9, 4), "unit": "GFLOP/s", "cores": ora.num_threads(), "kind": "oracle",
               "sample": f"{reps} oracle FP64 domain-wall hops (4D hop on all {Ls} slices, {Vh} even sites) "
                         f"in {el:.1f} s",
               "dw_apply_s": round(1.0 / rate_d, 3),
               "dw_apply_sample": f"{reps_d} applications of the full D_DW of Eq. (2) in {el_d:.1f} s"}
    out = {"workload": "dwf_16x16x16x32_Ls16_M5_1.8_mf0.02", "hop": hop, "cg": res, "roofline": roof,
           "cpu_baseline": cpu,
           "bicgstab_f32_df": bicg, "mobius_b5_1.5_c5_0.5": mob,
           "note": "cg keys: inner precision, _df = double-float outer steps (else IEEE FP64)",
           "speedup_f16_vs_f64": round(res["f64"]["ms"] / res["f16"]["ms"], 3),
           "speedup_f32_vs_f64": round(res["f64"]["ms"] / res["f32"]["ms"], 3),
           "speedup_f16_df_vs_f64": round(res["f64"]["ms"] / res["f16_df"]["ms"], 3),
           "speedup_f32_df_vs_f64": round(res["f64"]["ms"] / res["f32_df"]["ms"], 3)}
    print(json.dumps(out), flush=True)


def run_batched(args):
    L, kappa = (24, 24, 24, 48), 0.124
    V = int(np.prod(L))
    Vh = V // 2
    U = inputs.gauge_field(L, 0.2, 4)
    x0, b = inputs.point_sources(L, 0)
    dev = torch.device("cuda", 0)
    g = qcd.Gauge.load(torch.from_numpy(U).to(dev), L, BC, recon=12)
    f = qcd.wilson(kappa)
    bd = torch.from_numpy(b).to(dev)
    # 12-rhs stencil vs 12 single-rhs stencils (FP32, internal layout)
    nb12 = qcd.field_bytes(g, f, "f32", 12)
    a12 = torch.empty(nb12, dtype=torch.uint8, device=dev)
    o12 = torch.empty(nb12, dtype=torch.uint8, device=dev)
    qcd.field_pack(g, f, "f32", 1, bd, a12, nrhs=12)
    ms12 = _time_launches(lambda: qcd.dslash(g, f, "D_EO", a12, o12, prec="f32", nrhs=12, layout=qcd.INTERNAL))
    if args.profile not in ("none", "cg"):  # ncu: profile 3 launches of the 12-rhs hop (tuned above)
        pp = args.profile_prec if args.profile_prec in ("f32", "f16") else "f32"
        if pp != "f32":
            a12 = torch.empty(qcd.field_bytes(g, f, pp, 12), dtype=torch.uint8, device=dev)
            o12 = torch.empty_like(a12)
            qcd.field_pack(g, f, pp, 1, bd, a12, nrhs=12)
            _time_launches(lambda: qcd.dslash(g, f, "D_EO", a12, o12, prec=pp, nrhs=12, layout=qcd.INTERNAL))
        torch.cuda.profiler.start()
        for _ in range(3):
            qcd.dslash(g, f, "D_EO", a12, o12, prec=pp, nrhs=12, layout=qcd.INTERNAL)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(f"profile batched hop ({pp}) done", flush=True)
        return
    # the 12-rhs stencil in FP16 (the tuner's choice among its launch shapes, which include
    # one direction on the tensor cores)
    nb16 = qcd.field_bytes(g, f, "f16", 12)
    a16 = torch.empty(nb16, dtype=torch.uint8, device=dev)
    o16 = torch.empty(nb16, dtype=torch.uint8, device=dev)
    qcd.field_pack(g, f, "f16", 1, bd, a16, nrhs=12)
    ms16 = _time_launches(lambda: qcd.dslash(g, f, "D_EO", a16, o16, prec="f16", nrhs=12, layout=qcd.INTERNAL))
    del a16, o16
    nb1 = qcd.field_bytes(g, f, "f32", 1)
    ms1 = _time_launches(lambda: qcd.dslash(g, f, "D_EO", a12[:nb1], o12[:nb1], prec="f32",
                                            layout=qcd.INTERNAL))
    alg12 = Vh * (8 * 48 + 12 * 192)
    kw = dict(method=qcd.BICGSTAB, tol=1e-10, inner="f32", use_graph=True, graph_chunk=32,
              delta=(args.delta or 1e-5), outer=args.outer)
    x = torch.zeros_like(bd)
    qcd.solve(g, f, bd, x, nrhs=12, **kw)  # warm-up
    x.zero_()
    if args.profile == "cg":  # ncu launch list: one warmed-up batched solve
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        info, _ = qcd.solve(g, f, bd, x, nrhs=12, **kw)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(f"profile batched solve done: {[i['iters'] for i in info]}", flush=True)
        return
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info, _ = qcd.solve(g, f, bd, x, nrhs=12, **kw)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    xk = torch.zeros_like(bd[0])
    qcd.solve(g, f, bd[0].contiguous(), xk, **kw)  # warm-up of the single-rhs path (tuning, graphs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    iters_seq = []
    for k in range(12):
        xk = torch.zeros_like(bd[k])
        ik, _ = qcd.solve(g, f, bd[k].contiguous(), xk, **kw)
        iters_seq.append(ik[0]["iters"])
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    peak = _peak()
    roof = {"bound": "hbm", "kernel": "12-rhs D_eo, FP32 12-real", "achieved": round(alg12 / ms12 / 1e6, 1),
            "peak": peak, "unit": "GB/s", "frac": round(alg12 / ms12 / 1e6 / peak, 4), "algorithmic_bytes": alg12,
            "traffic": _traffic("batched_hop12_f32"), "note": "peak of measured copy bandwidth; 8 x 48 B links per site + 12 x (96 + 96) B"}
    cpu = None
    if not getattr(args, "no_cpu_baseline", False):
        from oracle import oracle as ora

        par = ora.parity(L)
        src = b[0].copy()
        src[par == 0] = 0
        rate, reps, el = _cpu_rate(lambda: ora.hop(L, BC, U, src, out_parity=0), metrics.HOP_FLOP_SITE * Vh)
        cpu = {"value": round(rate / 1e9, 4), "unit": "GFLOP/s", "cores": ora.num_threads(), "kind": "oracle",
               "sample": f"{reps} oracle FP64 D_eo applications to one right-hand side ({Vh} sites) in {el:.1f} s"}
    out = {"workload": "wilson_24x24x24x48_kappa0.124_12pointsources", "x0": x0, "roofline": roof,
           "cpu_baseline": cpu,
           "dslash12_ms": round(ms12, 4), "dslash12_gflops": round(metrics.HOP_FLOP_SITE * Vh * 12 / ms12 / 1e6, 1),
           "dslash12_gbs": round(alg12 / ms12 / 1e6, 1), "dslash12_frac": round(alg12 / ms12 / 1e6 / _peak(), 4),
           "dslash1_x12_ms": round(12 * ms1, 4), "dslash12_f16_ms": round(ms16, 4),
           "solve12_s": round(t_batch, 4), "solve_12x1_s": round(t_seq, 4),
           "speedup_batched": round(t_seq / t_batch, 3),
           "iters": [i["iters"] for i in info], "iters_seq": iters_seq,
           "max_true_resid": max(i["true_resid"] for i in info), "outer": args.outer}
    print(json.dumps(out), flush=True)


def run_force(args):
    from paper_1712_01505_gb300.autograd import wilson_action

    L, kappa = (16, 16, 16, 16), 0.12
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.3, 5)
    phi = inputs.gaussian_source((V, 4, 3), 0)
    dev = torch.device("cuda", 0)
    Ut = torch.from_numpy(U).to(dev)
    pt = torch.from_numpy(phi).to(dev)
    times = []
    for rep in range(4):
        u = Ut.clone().requires_grad_(True)
        S = wilson_action(u, pt, kappa, L, BC, tol=1e-10, inner="f32")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.backward()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    g = qcd.Gauge.load(Ut, L, BC)
    f = qcd.wilson(kappa)
    X = torch.from_numpy(inputs.gaussian_source((V, 4, 3), 1)).to(dev)
    out_t = torch.empty((4, V, 3, 3, 2), dtype=torch.float64, device=dev)
    ms = _time_launches(lambda: qcd.force(g, f, X, pt, out_t))
    if args.profile != "none":  # ncu: profile 3 launches of the force kernel
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        for _ in range(3):
            qcd.force(g, f, X, pt, out_t)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print("profile force done", flush=True)
        return
    # molecular dynamics of the even-odd action: one force evaluation (two mixed solves to 1e-10,
    # qcd_force_eo, qcd_force_project) and one leapfrog step (force + link and momentum updates)
    from paper_1712_01505_gb300 import hmc

    md = hmc.EOPseudofermionMD(L, kappa, pt, tol=1e-10)
    P = torch.from_numpy(inputs.su3_momenta((4, V), 2)).to(dev)
    Fm, _ = md.force(Ut)  # warm-up (tuning, workspace, graphs)
    t_force = []
    for rep in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        md.force(Ut, Fm)
        torch.cuda.synchronize()
        t_force.append(time.perf_counter() - t0)
    Uc, Pc = Ut.clone(), P.clone()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h0, h1 = md.leapfrog(Uc, Pc, 0.02, 1)
    torch.cuda.synchronize()
    t_step = time.perf_counter() - t0
    ms_eo = _time_launches(lambda: qcd.force_eo(g, f, X, pt, out_t))
    ms_proj = _time_launches(lambda: qcd.force_project(g, out_t, Fm))
    ms_link = _time_launches(lambda: qcd.link_update(Uc, Pc, 0.02))
    # the force kernel reads X and eta at a site and its neighbours (2 x 192 B per site from HBM)
    # and writes 4 links x 144 B; about 250 FP64 flop per link: FP64-bound on this GPU
    fp64_peak = _fp64_peak_tflops()
    force_flop = 4 * V * 250
    roof = {"bound": "alu", "kernel": "force outer product (k_force), FP64",
            "achieved": round(force_flop / ms / 1e9, 4), "peak": round(fp64_peak, 4), "unit": "TFLOP/s",
            "frac": round(force_flop / ms / 1e9 / fp64_peak, 4), "traffic": _traffic("force_kernel"),
            "hbm_frac": round(V * (2 * 192 + 4 * 144) / ms / 1e6 / _peak(), 4),
            "note": "peak = cuBLAS DGEMM 4096^3 measured in this run; ~250 FP64 flop per link"}
    cpu = None
    if not getattr(args, "no_cpu_baseline", False):
        from oracle import oracle as ora

        Xh = inputs.gaussian_source((V, 4, 3), 1)
        rate, reps, el = _cpu_rate(lambda: ora.wilson_force(L, BC, kappa, Xh, phi), 1.0)
        cpu = {"value": round(rate, 4), "unit": "force evaluations/s", "cores": ora.num_threads(), "kind": "oracle",
               "sample": f"{reps} oracle FP64 force outer products on 16^4 in {el:.1f} s",
               "gpu_kernel_per_s": round(1e3 / ms, 1)}
    out = {"workload": "force_wilson_16x16x16x16_kappa0.12", "roofline": roof, "cpu_baseline": cpu,
           "backward_ms": round(min(times[1:]) * 1e3, 3),
           "force_kernel_ms": round(ms, 4),
           "force_kernel_gbs": round(V * (2 * 192 + 4 * 144) / ms / 1e6, 1),
           "md": {"force_eval_ms": round(min(t_force) * 1e3, 3),
                  "leapfrog_step_ms": round(t_step * 1e3, 3),
                  "force_eo_ms": round(ms_eo, 4), "force_project_ms": round(ms_proj, 4),
                  "link_update_ms": round(ms_link, 4), "dH_one_step_0.02": h1 - h0}}
    print(json.dumps(out), flush=True)


def run_dd(args):
    """Domain decomposition on one GPU: the 32^3 x 64 Wilson system (config of the bench line) cut
    into subdomains held by this process (faces exchanged by device copies while the interior is
    computed): the decomposed Mhat and BiCGStab against the single-domain ones."""
    from paper_1712_01505_gb300 import dd

    L, kappa = (32, 32, 32, 64), 0.125
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.2, 2)
    b = inputs.z2_source((V, 4, 3), 0)
    dev = torch.device("cuda", 0)
    f = qcd.wilson(kappa)
    g = qcd.Gauge.load(torch.from_numpy(U).to(dev), L, BC, recon=12)
    bd = torch.from_numpy(b).to(dev)
    out = {"workload": "dd_wilson_32x32x32x64_kappa0.125", "note": "subdomains of one process on one GPU"}
    if args.profile == "cg":  # ncu launch list: one warmed-up decomposed solve in two subdomains
        P = (1, 1, 1, 2)
        ids = [0, 1]
        D = dd.Decomposition(L, P, BC, ids, [dd.scatter_gauge(U, L, P, s) for s in ids], recon=12)
        bl = [torch.from_numpy(dd.scatter_spinor(b, L, P, s)).to(dev) for s in ids]
        xl = [torch.zeros_like(t_) for t_ in bl]
        D.solve(f, bl, xl, tol=1e-10, inner="f32", delta=1e-5)
        for t_ in xl:
            t_.zero_()
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        info, _ = D.solve(f, bl, xl, tol=1e-10, inner="f32", delta=1e-5)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(f"profile dd solve done: {info}", flush=True)
        D.free()
        return
    src = bd.clone()
    w = torch.empty_like(bd)
    ref = {}
    for prec in ("f32", "f64"):
        ref[prec] = _time_launches(lambda: qcd.dslash(g, f, "MHAT", src, w, prec=prec), n=10)
    kw = dict(method=qcd.BICGSTAB, tol=1e-10, inner="f32", delta=1e-5, outer="f64")
    x = torch.zeros_like(bd)
    qcd.solve(g, f, bd, x, **kw)
    x.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info1, _ = qcd.solve(g, f, bd, x, **kw)
    torch.cuda.synchronize()
    out["single"] = {"mhat_f32_ms": round(ref["f32"], 4), "mhat_f64_ms": round(ref["f64"], 4),
                     "solve_ms": round((time.perf_counter() - t0) * 1e3, 2), "iters": info1[0]["iters"]}
    g.free()
    # (1, 1, 1, 1): the decomposed solver on the undivided lattice (no faces to exchange), its
    # own cost against the single-domain solver's
    for P in ((1, 1, 1, 1), (1, 1, 1, 2), (1, 1, 2, 2), (2, 2, 2, 2)):
        ids = list(range(int(np.prod(P))))
        D = dd.Decomposition(L, P, BC, ids, [dd.scatter_gauge(U, L, P, s) for s in ids], recon=12)
        bl = [torch.from_numpy(dd.scatter_spinor(b, L, P, s)).to(dev) for s in ids]
        ol = [torch.empty_like(t) for t in bl]
        t = {p: _time_launches(lambda: D.dslash(f, "MHAT", bl, ol, prec=p), n=10) for p in ("f32", "f64")}
        xl = [torch.zeros_like(t_) for t_ in bl]
        D.solve(f, bl, xl, tol=1e-10, inner="f32", delta=1e-5)
        for t_ in xl:
            t_.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info, _ = D.solve(f, bl, xl, tol=1e-10, inner="f32", delta=1e-5)
        torch.cuda.synchronize()
        out["P" + "x".join(map(str, P))] = {"mhat_f32_ms": round(t["f32"], 4), "mhat_f64_ms": round(t["f64"], 4),
                                            "solve_ms": round((time.perf_counter() - t0) * 1e3, 2),
                                            "iters": info["iters"], "updates": info["outer_updates"],
                                            "true_resid": info["true_resid"]}
        D.free()
        del bl, ol, xl
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)


def run_workload(args):
    torch.cuda.set_device(0)
    {"dwf": run_dwf, "batched": run_batched, "force": run_force, "dd": run_dd}[args.workload](args)
