#!/usr/bin/env python
"""Benchmark of the enriched-FE ChFSI hot path on one GB300.

Workload (default): the 16-atom silicon-like cluster -- two conventional
diamond cells (a = 10.26 bohr) of Z = 14 nuclei, box padded by 10 bohr, graded
degree-4 mesh (37 x 25 x 25 cells, 1.52M nodes), 5 Slater enrichment
functions per atom (n_E = 80), N = 135 vectors, Chebyshev degree m = 40, local
potential = nuclear Coulomb + a seeded 32-term Gaussian perturbation.

One step = one pass of the whole hot path: Lanczos upper bound (10 steps),
the degree-m Chebyshev filter of (M^E)^-1 H^E, Cholesky-QR and Rayleigh-Ritz
with residuals.  `value` is the filter's algorithmic TFLOP/s over the whole
step (filter flops / step time); the FP64-mode step is timed beside it.

--impl reference times the FP64 CPU oracle (test infrastructure) on a
bounded sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

NL = 125
N_VEC = 135
M_DEG = 40


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="tf32x3", choices=["tf32x3", "fp32", "tf32", "fp64"])
    p.add_argument("--fp64-tail", type=int, default=2)
    p.add_argument("--fp64-engine", default="tensor", choices=["tensor", "dfma"],
                   help="engine of the FP64 parts of the mixed step (the FP64 comparison always uses dfma)")
    p.add_argument("--fp64-steps", type=int, default=2)
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-scf", action="store_true")
    p.add_argument("--no-batch", action="store_true")
    p.add_argument("--scf-steps", type=int, default=3)
    p.add_argument("--workload", default="si16", choices=["si16", "si16s", "hydrogen"])
    return p.parse_args()


def workload(name):
    if name == "si16":
        return W.si_cluster(), N_VEC, M_DEG
    if name == "si16s":  # coarser mesh of the same cluster (profiling captures)
        return W.si_cluster(h_min=1.6, h_max=4.0), N_VEC, M_DEG
    return W.hydrogen(), 8, 20


WORKLOAD_TEXT = {
    "si16": "16-atom Si-like cluster (Z=14, diamond a=10.26), graded degree-4 mesh",
    "si16s": "16-atom Si-like cluster (Z=14, diamond a=10.26), coarser graded degree-4 mesh (h 1.6-4.0 bohr)",
    "hydrogen": "hydrogen Z=1, 6x6x6 cells",
}


def filter_flops(n_cell, nnz, nE, N, m):
    """Algorithmic flops of m filter degrees: cell products 2*125^2*N per cell,
    four sparse enrichment products 2*nnz*N, H^ee and S^-1 products 2*nE^2*N each."""
    return float(m) * N * (2.0 * NL * NL * n_cell + 8.0 * nnz + 4.0 * nE * nE)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            return float(d.get("hbm_gbs", 6800.0)), "measured"
        except Exception:
            pass
    return 6800.0, "fallback"


def peaks_bf16():
    """Dense BF16 tensor peak for a kernel timed inside a long step: the measured sustained
    figure if present, else the fallback 1700 TFLOP/s."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            v = d.get("bf16_tflops_sustained", d.get("bf16_tflops"))
            if v:
                return float(v), "measured"
        except Exception:
            pass
    return 1700.0, "fallback (sustained)"


def clocks_start(dev):
    """Sample SM clocks, power and throttle reasons every 200 ms (nvidia-smi) while
    the timed region runs; the samples are parsed in memory."""
    try:
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200",
                              "-i", str(dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        return p
    except Exception:
        return None


def clocks_stop(p):
    if p is None:
        return None
    p.terminate()
    try:
        out, _ = p.communicate(timeout=5)
    except Exception:
        p.kill()
        out, _ = p.communicate()
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.strip().splitlines():
        c = [x.strip() for x in line.split(",")]
        if len(c) < 9:
            continue
        try:
            sm.append(float(c[1]))
            mx.append(float(c[2]))
        except ValueError:
            continue
        for n, v in zip(names, c[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
            "samples": len(sm)}


def cpu_sample(system, N, steps=None, min_seconds=10.0):
    """The oracle (FP64 NumPy) on a bounded sample: its elemental H~ apply over an
    8 x 8 x 8-cell corner window of the same graded mesh, same nuclei and potential,
    repeated for about ``min_seconds`` (or exactly ``steps`` applies).
    Returns (TFLOP/s, seconds per apply, description)."""
    from oracle.operators import Discretisation
    sub = dict(system)
    sub["breaks"] = [b[:9] for b in system["breaks"]]
    sub["funcs"] = []
    d = Discretisation(sub)
    X = W.random_block(sub, N, seed=21)
    flops = filter_flops(d.n_cell, 0, 0, N, 1)
    n = 0
    t = time.perf_counter()
    while True:
        d.apply_Htilde(X)
        n += 1
        el = time.perf_counter() - t
        if (steps is not None and n >= steps) or (steps is None and el >= min_seconds and n >= 3):
            break
    dt = el / n
    desc = (f"oracle elemental H~ apply (FP64 NumPy), N={N}, over an 8x8x8-cell corner window "
            f"({d.n_cell} cells) of the same mesh and potential; {n} applies, {el:.1f} s; "
            "TFLOP/s by the same algorithmic count")
    return flops / dt / 1e12, dt, desc


def batch_section(P, torch, stream, n_sys=8, m=20, steps=3):
    import math
    rng = np.random.default_rng(5)
    Gs, Xs, Ns, flops, tiles, nodes = [], [], [], 0.0, [], []
    for i in range(n_sys):
        na = int(rng.integers(1, 7))
        s = W.random_cluster(na, [1, 6, 8, 14], seed=500 + i, h_min=1.2, h_max=4.0, pad=7.0)
        G = P.System(s)
        G.set_potential_analytic()
        ne = float(np.sum(s["Z"]))
        N = int(math.ceil(0.6 * ne)) + 8
        X = torch.from_numpy(W.initial_block(s, N, seed=1)).cuda()
        G.rayleigh_ritz(X)
        tile, _ = G.autotune(N, "tf32x3")
        Gs.append(G)
        Xs.append(X)
        Ns.append(N)
        tiles.append(tile)
        nodes.append(G.n_nodes)
        flops += filter_flops(G.n_cells, G.n_coupling, G.n_enrich, N, m)
    a, b, a0 = [], [], []
    for G, X in zip(Gs, Xs):
        e, _ = G.rayleigh_ritz(X)
        a.append(e.max())
        a0.append(e.min())
        b.append(G.upper_bound(X[:, -1].contiguous(), 10))
    B = P.Batch(Gs)
    out = {}
    for mode in (True, False):
        Xw = [x.clone() for x in Xs]
        B.chfsi_step(Xw, m, a, b, a0, precision="tf32x3", fp64_tail=2, graph=mode)   # warm-up / recording
        torch.cuda.synchronize()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        s0.record(stream)
        for _ in range(steps):
            B.chfsi_step(Xw, m, a, b, a0, precision="tf32x3", fp64_tail=2, graph=mode)
        s1.record(stream)
        torch.cuda.synchronize()
        out[mode] = (time.perf_counter() - t0) / steps
    nn, kn = B.graph_nodes()
    B.close()
    return {"systems": n_sys, "nodes": nodes, "N": Ns, "m": m, "precision": "tf32x3, FP64 tail 2",
            "graph_s_per_step": out[True], "sequential_s_per_step": out[False],
            "graph_speedup": out[False] / out[True], "graph_tflops": flops / out[True] / 1e12,
            "graph_nodes": nn, "graph_kernel_nodes": kn, "autotuned_tiles": tiles,
            "step": "one filter step of every system (no Rayleigh-Ritz), host wall clock incl. graph launch"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    system, N, m = workload(args.workload)
    from oracle.operators import Discretisation  # noqa: F401
    for _ in range(args.warmup):
        cpu_sample(system, N, steps=1)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, dt, desc = cpu_sample(system, N, steps=1)
        vals.append((v, dt))
    tot = time.perf_counter() - t0
    value = statistics.median(v for v, _ in vals)
    cores = len(os.sched_getaffinity(0))
    line = {"impl": "reference", "metric": "chfsi_filter_tflops", "value": value, "unit": "TFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "si16: 16-atom Si-like cluster, 1.52M-node graded degree-4 mesh, N=135, m=40",
                       "sample": desc},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__ as g
    g.build()
    import paper_1610_02121_gb300 as P
    system, N, m = workload(args.workload)
    t_setup = time.perf_counter()
    G = P.System(system)
    G.set_potential_analytic()
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    X0 = torch.from_numpy(W.initial_block(system, N, seed=1)).cuda()
    v0 = torch.from_numpy(W.lanczos_start(system)).cuda()
    X = X0.clone()
    eps, res = G.rayleigh_ritz(X)
    X_start = X.clone()
    eps_start = eps.copy()
    stream = torch.cuda.current_stream()

    def one_step(Xb, eps_prev, prec):
        b = G.upper_bound(v0, 10)
        G.chfsi_step(Xb, m, eps_prev.max(), b, eps_prev.min(), precision=prec,
                     fp64_tail=(args.fp64_tail if prec != "fp64" else 0))
        e, r = G.rayleigh_ritz(Xb)
        return e, r, b

    def timed(prec, warm, steps, timing=False, engine=None):
        G.set_fp64_engine(engine or (args.fp64_engine if prec != "fp64" else "dfma"))
        Xb = X_start.clone()
        e = eps_start.copy()
        for _ in range(warm):
            e, r, b = one_step(Xb, e, prec)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        if timing:
            G.enable_timing(True)
            G.kernel_stats(reset=True)
            G.kernel_stats_fp64(reset=True)
        l0 = P.launch_count()
        clk = clocks_start(local) if timing else None
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(steps):
            e, r, b = one_step(Xb, e, prec)
        s1.record(stream)
        torch.cuda.synchronize()
        ms = s0.elapsed_time(s1) / steps
        clocks = clocks_stop(clk) if timing else None
        launches = P.launch_count() - l0
        stats = (G.kernel_stats(reset=True), G.kernel_stats_fp64(reset=True)) if timing else None
        G.enable_timing(False)
        if dist is not None:
            t = torch.tensor([ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms, e, r, b, launches // max(steps, 1), clocks, stats

    prec = args.precision
    ms, eps_m, res_m, b, launches, clocks, stats = timed(prec, args.warmup, args.steps, timing=True)
    flops_step = filter_flops(G.n_cells, G.n_coupling, G.n_enrich, N, m)
    value = world * flops_step / (ms * 1e-3) / 1e12
    # the two tensor-core kernels of the step: the mixed filter's cell products and the
    # FP64 engine (tail degrees, Cholesky-QR, Rayleigh-Ritz); the roofline object
    # describes the one with the larger share of the step time, the other sits beside it
    (n_launch, k_ms, cellcols), (oz_launch, oz_ms, oz_flops) = stats
    s_el = {"fp64": 8, "fp32": 4, "tf32": 4, "tf32x3": 4, "bf16": 2}[prec]
    h_bytes = G.n_cells * NL * NL * s_el
    v_bytes = 2.0 * G.n_nodes * N * s_el
    frac_cells = cellcols / float(G.n_cells * N)
    alg_bytes = (h_bytes + v_bytes) * frac_cells
    alg_flops = 2.0 * NL * NL * cellcols
    hbm_peak, peak_src = peaks()
    if prec in ("fp32", "fp64"):
        # SIMT-bound: FP32 FFMA peak from 152 SMs x 128 lanes x 2 flop x 2.07 GHz; FP64 from the measured DGEMM
        peak = 80.5 if prec == "fp32" else 1.05
        achieved = alg_flops / (k_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": f"k_cell_apply<{'float' if prec == 'fp32' else 'double'}>",
                "launches": n_launch, "avg_launch_ms": k_ms / max(n_launch, 1),
                "algorithmic_gbs": alg_bytes / (k_ms * 1e-3) / 1e9,
                "peak_source": "derived from unit counts and max clock" if prec == "fp32" else "measured DGEMM"}
    else:
        achieved = alg_bytes / (k_ms * 1e-3) / 1e9
        # DRAM traffic of one launch from the ncu capture of this kernel on the si16s mesh
        # (249 MB for 1,053 cells at N = 135: 237 KB per cell), scaled by the cells per launch
        cells_per_launch = cellcols / float(max(n_launch, 1) * N)
        traffic = 236.7e3 * cells_per_launch if (prec == "tf32x3" and N == 135) else None
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                "traffic": traffic, "traffic_source": "ncu dram bytes of the si16s capture, scaled by cells per launch",
                "algorithmic_bytes_per_launch": alg_bytes / max(n_launch, 1),
                "kernel": "k_cell_tc3<%s>" % ("true" if prec == "tf32x3" else "false"),
                "launches": n_launch, "algorithmic_tflops": alg_flops / (k_ms * 1e-3) / 1e12,
                "avg_launch_ms": k_ms / max(n_launch, 1), "peak_source": peak_src}
    roof_oz = None
    if oz_launch > 0 and oz_ms > 0:
        bf16_peak, bf16_src = peaks_bf16()
        oz_tf = oz_flops / (oz_ms * 1e-3) / 1e12
        # DRAM traffic per launch: ncu dram bytes of every k_oz launch of one si16s step (CELL 0.90 GB,
        # symmetric Gram 2.48 GB, A^T B Gram 3.79 GB, rotation 2.73 GB), weighted by the step's mix
        # (24 / 1 / 2 / 4 launches) and scaled to si16 by the rows and cells processed (x 2.72)
        oz_traffic = 3.73e9 if (args.workload == "si16" and N == 135 and m == 40) else None
        roof_oz = {"bound": "tensor", "achieved": 28.0 * oz_tf, "peak": bf16_peak, "unit": "TFLOP/s",
                   "frac": 28.0 * oz_tf / bf16_peak, "traffic": oz_traffic,
                   "traffic_source": "ncu dram bytes per mode on si16s, step mix, scaled x2.72 to si16",
                   "kernel": "k_oz (FP64-grade products)",
                   "launches": oz_launch, "avg_launch_ms": oz_ms / oz_launch, "fp64_grade_tflops": oz_tf,
                   "vs_fp64_dgemm_peak": oz_tf / 1.05,
                   "note": "achieved = 28 BF16 digit products per FP64 product x algorithmic FP64 flops / time",
                   "peak_source": bf16_src}
    roof_cells = roof
    if roof_oz is not None and oz_ms > k_ms:
        roof, roof_other = roof_oz, roof_cells
    else:
        roof, roof_other = roof_cells, roof_oz
    line = {"metric": "chfsi_filter_tflops", "value": value, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": prec if prec != "fp64" else "f64",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: " + WORKLOAD_TEXT[args.workload],
                       "nodes": G.n_nodes, "cells": G.n_cells, "n_enrich": G.n_enrich, "n_coupling": G.n_coupling, "N": N, "m": m,
                       "fp64_tail": args.fp64_tail if prec != "fp64" else 0,
                       "fp64_engine": args.fp64_engine if prec != "fp64" else "dfma",
                       "l2": "vector blocks (>= 0.8 GB) and cell matrices exceed the 129 MB L2",
                       "step": "Lanczos bound (10) + degree-m filter + CholQR + Rayleigh-Ritz",
                       "filter_flops_per_step": flops_step, "setup_s": t_setup},
            "s_per_step": ms * 1e-3, "gpu_launches": launches, "roofline": roof}
    if roof_other is not None:
        line["roofline_other_kernel"] = roof_other
    line["kernel_ms_per_step"] = {"k_cell_tc3": k_ms / args.steps, "k_oz": oz_ms / args.steps}
    line["shifted_cholqr_passes_total"] = G.rr_shifted_passes()
    if clocks:
        line["clocks"] = clocks
    # FP64 mode of the same step
    if not args.no_fp64 and prec != "fp64":
        ms64, eps64, res64, _, _, _, _ = timed("fp64", 1, args.fp64_steps, engine="dfma")
        _, eps_chk, _, _, _, _, _ = timed(prec, 1, args.fp64_steps)
        ms64t, eps64t, _, _, _, _, _ = timed("fp64", 1, args.fp64_steps, engine="tensor")
        line["fp64"] = {"ms_per_step": ms64, "tflops": flops_step / (ms64 * 1e-3) / 1e12,
                        "engine": "dfma (plain FP64)",
                        "speedup_mixed_vs_fp64": ms64 / ms,
                        "max_abs_eig_diff_vs_fp64_Ha": float(np.abs(eps_chk - eps64).max()),
                        "steps_compared": 1 + args.fp64_steps}
        line["fp64_tensor_engine"] = {"ms_per_step": ms64t, "tflops": flops_step / (ms64t * 1e-3) / 1e12,
                                      "max_abs_eig_diff_vs_dfma_Ha": float(np.abs(eps64t - eps64).max())}
    # end to end through the public API with host buffers
    if not args.no_e2e:
        Xh = X_start.cpu().pin_memory()
        Xd = torch.empty_like(X_start)
        e = eps_start.copy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            Xd.copy_(Xh, non_blocking=True)
            e, r, _ = one_step(Xd, e, prec)
            Xh.copy_(Xd, non_blocking=True)
        torch.cuda.synchronize()
        te = (time.perf_counter() - t0) / args.steps
        nb = X_start.numel() * 8
        line["e2e"] = {"value": world * flops_step / te / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": nb,
                       "d2h_bytes_per_step": nb + 2 * 8 * N, "ms_per_step": te * 1e3}
    # full SCF iterations (Sec. V) on the same system: V_eff from rho_in (Hartree
    # solve + LDA), bound, filter pass, Rayleigh-Ritz, occupations, density,
    # Hartree of rho_out, energies, Anderson mixing
    if not args.no_scf:
        G.set_fp64_engine(args.fp64_engine)
        ne = float(np.sum(system["Z"]))
        occ0, _ = P._lib.fermi(eps_start, ne, 500 * P._lib.KB_HA_PER_K)
        rho_in = G.density(X_start, occ0)
        w = G.qpoints()[:, 3]
        rho_in *= ne / float((w * rho_in).sum())
        rho_out = torch.empty_like(rho_in)
        Xs = X_start.clone()
        G.scf_init(ne)
        tail = args.fp64_tail if prec != "fp64" else 0
        r0 = G.scf_step(Xs, rho_in, rho_out, m, precision=prec, fp64_tail=tail)   # warm-up
        torch.cuda.synchronize()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        hist = []
        for _ in range(args.scf_steps):
            hist.append(G.scf_step(Xs, rho_in, rho_out, m, precision=prec, fp64_tail=tail))
        s1.record(stream)
        torch.cuda.synchronize()
        ms_scf = s0.elapsed_time(s1) / max(args.scf_steps, 1)
        line["scf"] = {"s_per_iteration": ms_scf * 1e-3, "iterations_timed": args.scf_steps,
                       "n_electrons": ne, "kT_K": 500.0, "anderson_stages": 5, "mixing": 0.5,
                       "filter": f"one degree-{m} pass, {prec}", "n_qpoints": G.n_qpoints,
                       "poisson_correction_steps": [h["poisson_steps"] for h in hist],
                       "total_energy_Ha": [h["total"] for h in [r0] + hist],
                       "drho": [h["drho"] for h in [r0] + hist],
                       "start": "density of the Rayleigh-Ritz-rotated atomic-orbital block, renormalised to N_e"}
    # many small systems (1-6 atoms, Z in {1, 6, 8, 14}, own graded meshes, N = ceil(0.6 N_e) + 8):
    # one ChFSI filter step of every system as one CUDA graph vs the same steps launched
    # one system after another; column tiles of the cell kernel picked by the autotuner
    if not args.no_batch and rank == 0:
        line["batch"] = batch_section(P, torch, stream)
    if not args.no_cpu and rank == 0 and world == 1:
        v, dt, desc = cpu_sample(system, N)
        line["cpu_baseline"] = {"value": v, "unit": "TFLOP/s", "cores": len(os.sched_getaffinity(0)),
                                "kind": "oracle", "sample": desc}
    line["eigs_head"] = [float(x) for x in eps_m[:5]]
    line["max_resid"] = float(res_m.max())
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
