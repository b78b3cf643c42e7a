#!/usr/bin/env python
"""Benchmark of the enriched-FE ChFSI hot path on one GB300.

Workload (default, ``si280``): the paper's 280-atom silicon cluster -- a cube
cut of 3 x 3 x 3 conventional diamond cells (a = 10.26 bohr) including the
boundary atoms, Z = 14 (3920 electrons), box padded by 10 bohr, graded degree-4
mesh of 36^3 cells (3,048,625 nodes), 5 Slater enrichment functions per atom
(n_E = 1400), N = 2200 vectors, Chebyshev degree m = 40, local potential =
nuclear Coulomb + a seeded 32-term Gaussian perturbation.  ``si16`` is the
16-atom cluster (1.52M nodes, N = 135).

One step = one pass of the whole hot path: Lanczos upper bound (10 steps),
the degree-m Chebyshev filter of (M^E)^-1 H^E (mixed precision: 3-term TF32
tensor-core cell products, FP32 coupling, the last 2 degrees in FP64),
Cholesky-QR and Rayleigh-Ritz (Ritz values; the residuals are formed once
after the timed steps).  `value` is the filter's algorithmic TFLOP/s over the
whole step (filter flops / step time).  Beside it: the FP64-mode step, the
step through the C ABI with host buffers (e2e), and full SCF iterations.

--impl reference times the FP64 CPU oracle (test infrastructure) on a
bounded sample of the same workload.
"""
import argparse
import json
import math
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
WORKLOADS = {
    # name: (generator, N, m, text)
    "si280": (W.si280, 2200, 40,
              "si280: 280-atom Si-like cluster (cube cut of 3x3x3 diamond cells, Z=14, 3920 e-), "
              "graded degree-4 mesh 36^3 cells"),
    "si16": (W.si_cluster, 135, 40, "si16: 16-atom Si-like cluster (Z=14, diamond a=10.26), graded degree-4 mesh"),
    "si16s": (lambda: W.si_cluster(h_min=1.6, h_max=4.0), 135, 40,
              "si16s: 16-atom Si-like cluster, coarser graded degree-4 mesh (h 1.6-4.0 bohr)"),
    "hydrogen": (W.hydrogen, 8, 20, "hydrogen Z=1, 6x6x6 cells"),
    # the 280-atom block width on a small mesh (profiling case that fits a full ncu capture)
    "co2200": (W.carbon_monoxide, 2200, 4, "C-O pair mesh (49,005 nodes) with an N = 2200 block"),
}
# the largest blocks are generated on the device (a seeded torch generator);
# smaller ones by workloads.initial_block (NumPy PCG64)
DEVICE_INIT_BYTES = 4 << 30


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None, help="timed steps (default: 2 for si280, 5 otherwise)")
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="tf32x3", choices=["tf32x3", "fp32", "tf32", "fp64"])
    p.add_argument("--fp64-tail", type=int, default=2)
    p.add_argument("--fp64-engine", default="tensor", choices=["tensor", "dfma"],
                   help="engine of the FP64 parts of the mixed step")
    p.add_argument("--fp64-steps", type=int, default=1)
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-scf", action="store_true")
    p.add_argument("--dof-degree", action="store_true",
                   help="also run the enriched-vs-classical DoF x degree comparison (bare Z = 14 nucleus)")
    p.add_argument("--heavy-z", action="store_true", help="also run the heavy-Z multi-pass filter case (Z = 79 dimer)")
    p.add_argument("--converged", default="co", choices=["co", "si16", "none"],
                   help="system of the time-to-converged-SCF comparison (plain FP64 against mixed)")
    p.add_argument("--batch", action="store_true", help="also time the batched small systems (CUDA graph)")
    p.add_argument("--scf-steps", type=int, default=None, help="timed SCF iterations (default: 1 for si280, 3)")
    p.add_argument("--workload", default="si280", choices=sorted(WORKLOADS))
    a = p.parse_args()
    big = a.workload == "si280"
    if a.steps is None:
        a.steps = 2 if big else 5
    if a.scf_steps is None:
        a.scf_steps = 1 if big else 3
    return a


def filter_flops(n_cell, nnz, nE, N, m):
    """Algorithmic flops of m filter degrees: cell products 2*125^2*N per cell,
    four sparse enrichment products 2*nnz*N, H^ee and S^-1 products 2*nE^2*N each."""
    return float(m) * N * (2.0 * NL * NL * n_cell + 8.0 * nnz + 4.0 * nE * nE)


def _peaks_file():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            return json.load(open(path))
        except Exception:
            return None
    return None


def peaks():
    d = _peaks_file()
    if d and d.get("hbm_gbs"):
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def peaks_bf16():
    """Dense BF16 tensor peak for a kernel timed inside a long step: the measured sustained
    figure if present, else the fallback 1700 TFLOP/s."""
    d = _peaks_file()
    if d:
        v = d.get("bf16_tflops_sustained", d.get("bf16_tflops"))
        if v:
            return float(v), "measured"
    return 1700.0, "fallback (sustained)"


def clocks_start(dev):
    """Sample SM clocks, power and throttle reasons every 200 ms (nvidia-smi) while
    the timed region runs; the samples are parsed in memory."""
    try:
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        return subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200",
                                 "-i", str(dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
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


# ------------------------------------------------------------------------- CPU oracle sample
def oracle_window(system, cells=4):
    """A window of cells x cells x cells cells at the middle of the mesh with the
    enrichment functions whose support meets it (same nuclei and potential):
    the bounded sample the CPU oracle is timed on."""
    nc = [len(b) - 1 for b in system["breaks"]]
    lo = [max(0, n // 2 - cells // 2) for n in nc]
    sub = dict(system)
    sub["breaks"] = [b[l:l + cells + 1] for b, l in zip(system["breaks"], lo)]
    blo = np.array([b[0] for b in sub["breaks"]])
    bhi = np.array([b[-1] for b in sub["breaks"]])
    keep = []
    for f in system["funcs"]:
        R = system["atoms"][f["atom"]]
        if np.sqrt(np.sum(np.maximum(0.0, np.maximum(blo - R, R - bhi)) ** 2)) < f["r0"] * (1.0 + 1.0 / f["t"]):
            keep.append(f)
    sub["funcs"] = keep
    return sub


def cpu_sample(system, N, steps=None, min_seconds=10.0):
    """The oracle (FP64 NumPy) on a bounded sample: its elemental H~ apply (cell
    products, enrichment coupling, block-wise overlap inverse) over a 4x4x4-cell
    window at the middle of the same mesh with the enrichment functions that meet
    it, repeated for about ``min_seconds`` (or exactly ``steps`` applies).
    Returns (TFLOP/s, seconds per apply, description)."""
    from oracle.operators import Discretisation
    sub = oracle_window(system)
    d = Discretisation(sub)
    X = W.random_block(sub, N, seed=21)
    nnz = int(d.Mec_global.nnz) if d.nE > 0 else 0
    flops = filter_flops(d.n_cell, nnz, len(sub["funcs"]), N, 1)
    n = 0
    t = time.perf_counter()
    while True:
        d.apply_Htilde(X)
        n += 1
        el = time.perf_counter() - t
        if (steps is not None and n >= steps) or (steps is None and el >= min_seconds and n >= 3):
            break
    dt = el / n
    desc = (f"oracle elemental H~ apply (FP64 NumPy: cell products, enrichment coupling, block-wise "
            f"overlap inverse), N={N}, over a 4x4x4-cell window at the middle of the same mesh ({d.n_cell} cells, "
            f"{len(sub['funcs'])} enrichment functions, {nnz} coupling nonzeros) with the same nuclei and "
            f"potential; {n} applies, {el:.1f} s; TFLOP/s by the same algorithmic count")
    return flops / dt / 1e12, dt, desc


# ------------------------------------------------------------------------- batched small systems
def batch_section(P, torch, stream, n_sys=8, m=20, steps=3):
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
        t0 = time.perf_counter()
        for _ in range(steps):
            B.chfsi_step(Xw, m, a, b, a0, precision="tf32x3", fp64_tail=2, graph=mode)
        torch.cuda.synchronize()
        out[mode] = (time.perf_counter() - t0) / steps
    nn, kn = B.graph_nodes()
    B.close()
    return {"systems": n_sys, "nodes": nodes, "N": Ns, "m": m, "precision": "tf32x3, FP64 tail 2",
            "graph_s_per_step": out[True], "sequential_s_per_step": out[False],
            "graph_speedup": out[False] / out[True], "graph_tflops": flops / out[True] / 1e12,
            "graph_nodes": nn, "graph_kernel_nodes": kn, "autotuned_tiles": tiles,
            "step": "one filter step of every system (no Rayleigh-Ritz), host wall clock incl. graph launch"}


# ------------------------------------------------------------------------- converged SCF
CONVERGED = {
    # name: (generator, N, m, Anderson mixing, stages, atoms text)
    "co": (W.carbon_monoxide, 12, 24, 0.5, 5, "C-O pair (Z = 6, 8; 14 electrons; 49,005 nodes, 10 enrichment functions)"),
    "si16": (W.si_cluster, 135, 40, 0.2, 8, "si16: 16-atom Si-like cluster (224 electrons; 1.52M nodes, 80 enrichment "
                                             "functions)"),
}


def converged_scf_section(P, torch, prec, which="co", tol_e_atom=1e-7, tol_rho=3e-5, max_it=150):
    """Time to a converged SCF (Sec. V), plain FP64 (DFMA) against the mixed mode
    (tensor-core filter, FP64 tail degrees, FP64-grade Rayleigh-Ritz on the
    tensor cores): same start (the density of the Rayleigh-Ritz-rotated start
    block with Fermi occupations), one degree-m filter pass per iteration,
    Anderson mixing, T = 500 K; converged when |dE| < tol_e_atom per atom and
    ||rho_out - rho_in|| < tol_rho (the mixed mode's FP32-grade orbital values
    put its density noise near 1e-5)."""
    gen, N, m, beta, n_hist, text = CONVERGED[which]
    s = gen()
    G = P.System(s)
    G.set_potential_analytic()
    ne = float(np.sum(s["Z"]))
    tol_e = tol_e_atom * len(s["Z"])
    X0 = torch.from_numpy(W.initial_block(s, N, seed=1)).cuda()
    G.set_fp64_engine("dfma")
    eps0, _ = G.rayleigh_ritz(X0, residuals=False)
    occ0, _ = P._lib.fermi(eps0, ne, 500 * P._lib.KB_HA_PER_K)
    rho0 = G.density(X0, occ0)
    w = G.qpoints()[:, 3]
    rho0 *= ne / float((w * rho0).sum())
    out = {}
    for label, p, eng in (("fp64", "fp64", "dfma"), ("mixed", prec, "tensor")):
        G.set_fp64_engine(eng)
        X = X0.clone()
        rho_in = rho0.clone()
        rho_out = torch.empty_like(rho_in)
        G.scf_init(ne, beta=beta, n_hist=n_hist)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e_prev, r, it = None, None, 0
        for it in range(1, max_it + 1):
            r = G.scf_step(X, rho_in, rho_out, m, precision=p, fp64_tail=0 if p == "fp64" else 2)
            if e_prev is not None and abs(r["total"] - e_prev) < tol_e and r["drho"] < tol_rho:
                break
            e_prev = r["total"]
        torch.cuda.synchronize()
        nocc = int(np.sum(r["occ"] > 0.5))
        out[label] = {"wall_s": time.perf_counter() - t0, "iterations": it, "converged": it < max_it,
                      "total_energy_Ha": r["total"], "drho": r["drho"],
                      "eig_head_Ha": [float(x) for x in r["eig"][:5]],
                      "homo_Ha": float(r["eig"][max(nocc - 1, 0)]), "precision": p, "fp64_engine": eng}
    G.close()
    na = len(s["Z"])
    return {"system": f"{text}, N = {N}, m = {m}, Anderson {n_hist} stages, mixing {beta}",
            "criterion": f"|dE| < {tol_e_atom:g} Ha per atom and ||rho_out - rho_in|| < {tol_rho:g}",
            "fp64": out["fp64"], "mixed": out["mixed"],
            "speedup_mixed_vs_fp64": out["fp64"]["wall_s"] / out["mixed"]["wall_s"],
            "abs_dE_per_atom_Ha": abs(out["mixed"]["total_energy_Ha"] - out["fp64"]["total_energy_Ha"]) / na}


# ------------------------------------------------------------------------- DoF x degree, heavy Z
def dof_degree_section(P, torch, Z=14.0, N=8, nconv=5, tol=1e-7, max_iter=150):
    """The enriched-vs-classical comparison of Sec. VI.B.1 on a case with a closed
    form: a bare nucleus of charge Z (the Si-like core; -Z^2/(2n^2): 1s at -98 Ha,
    n = 2 at -24.5 Ha) in a 20-bohr box.  Enriched: 6^3 uniform cells with the
    hydrogenic 1s/2s/2p functions, filter degree 20; classical (n_E = 0): graded
    meshes refined to h_min at the nucleus, the degree scaled by sqrt(b / b_enriched)
    (the Chebyshev damping depends on the spectral width over the wanted gap).
    ChFSI in FP64 until the lowest five residuals are < tol; errors of the five
    lowest eigenvalues against the closed form, DoF (unknowns), degree, filter
    passes, wall time."""
    exact = np.array([-Z * Z / 2.0] + [-Z * Z / 8.0] * 4)
    rows, b_enr = [], None
    for enriched, h in [(True, None), (False, 0.2), (False, 0.1), (False, 0.05)]:
        s = W.bare_nucleus(Z=Z, enriched=enriched, h_min=h)
        G = P.System(s)
        G.set_potential_analytic()
        G.set_fp64_engine("dfma")
        X = torch.from_numpy(W.initial_block(s, N, seed=1)).cuda()
        v0 = torch.from_numpy(W.lanczos_start(s)).cuda()
        b = G.upper_bound(v0, 10)
        if enriched:
            b_enr = b
        m = 20 if enriched else int(math.ceil(20 * math.sqrt(b / b_enr)))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        eps, res, it, _ = G.solve(X, m, tol=tol, max_iter=max_iter, v0=v0, n_conv=nconv)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        dof = int(np.sum(~W.boundary_mask(s))) + G.n_enrich
        rows.append({"basis": "enriched (hydrogenic 1s/2s/2p)" if enriched else f"classical, h_min {h} bohr",
                     "dof": dof, "cells": G.n_cells, "upper_bound_Ha": b, "degree": m, "filter_passes": it,
                     "degree_x_passes": m * it, "wall_s": wall, "max_resid": float(np.max(res[:nconv])),
                     "max_abs_err_Ha": float(np.max(np.abs(eps[:nconv] - exact))),
                     "err_by_state_Ha": [float(x) for x in eps[:nconv] - exact]})
        G.close()
        del X
    return {"system": f"bare nucleus Z = {Z:g} in a 20-bohr box (closed form -Z^2/2n^2)", "N": N,
            "states_compared": "1s, 2s, 2p x 3", "runs": rows}


def heavy_z_section(P, torch, prec, passes_max=60, m=20, tol=1e-6):
    """Heavy-Z stand-in (Sec. VI.B.2: the gold clusters' multi-pass filter, 30
    passes of degree 20): two Z = 79 nuclei, Slater 1s/2s/2p enrichment, N = N_e/2
    + 20 = 99, bare nuclear potential; passes of a degree-m filter, each followed
    by Cholesky-QR and Rayleigh-Ritz, until the 79 lowest residuals are < tol."""
    s = W.gold_dimer()
    G = P.System(s)
    G.set_potential_analytic()
    out = {}
    for label, p, eng in (("fp64", "fp64", "dfma"), ("mixed", prec, "tensor")):
        G.set_fp64_engine(eng)
        X = torch.from_numpy(W.initial_block(s, 99, seed=1)).cuda()
        v0 = torch.from_numpy(W.lanczos_start(s)).cuda()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        eps, res, it, b = G.solve(X, m, tol=tol, max_iter=passes_max, v0=v0, n_conv=79, precision=p,
                                  fp64_tail=0 if p == "fp64" else 2)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        out[label] = {"passes": it, "wall_s": wall, "s_per_pass": wall / max(it, 1), "upper_bound_Ha": b,
                      "max_resid_79": float(np.max(res[:79])), "eig_head_Ha": [float(x) for x in eps[:3]],
                      "precision": p, "fp64_engine": eng}
    n_nodes, n_cells = G.n_nodes, G.n_cells
    G.close()
    return {"system": f"Au2-like dimer (Z = 79, 4.67 bohr), {n_nodes} nodes, {n_cells} cells, 10 enrichment functions",
            "N": 99, "degree": m, "tol": tol, "fp64": out["fp64"], "mixed": out["mixed"],
            "max_abs_eig_diff_Ha": float(np.max(np.abs(np.array(out["fp64"]["eig_head_Ha"]) -
                                                        np.array(out["mixed"]["eig_head_Ha"]))))}


# ------------------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    gen, N, m, text = WORKLOADS[args.workload]
    system = gen()
    for _ in range(args.warmup):
        cpu_sample(system, N, steps=1)
    vals = []
    t0 = time.perf_counter()
    desc = ""
    for _ in range(args.steps):
        v, dt, desc = cpu_sample(system, N, steps=1)
        vals.append(v)
    tot = time.perf_counter() - t0
    value = statistics.median(vals)
    cores = len(os.sched_getaffinity(0))
    line = {"impl": "reference", "metric": "chfsi_filter_tflops", "value": value, "unit": "TFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": text, "N": N, "m": m, "sample": desc},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------------- GPU arm
def initial_block(torch, system, G, N, seed=1):
    """X_0: unit vectors on the first min(N, n_E) enrichment coefficients (the atomic
    orbitals), seeded normal values on the interior nodes in the other columns."""
    if G.rows * N * 8 <= DEVICE_INIT_BYTES:
        return torch.from_numpy(W.initial_block(system, N, seed=seed)).cuda()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    X = torch.zeros((G.rows, N), dtype=torch.float64, device="cuda")
    k = min(N, G.n_enrich)
    idx = torch.arange(k, device="cuda")
    X[G.n_nodes + idx, idx] = 1.0
    if N > k:
        X[:G.n_nodes, k:] = torch.randn((G.n_nodes, N - k), generator=gen, dtype=torch.float64, device="cuda")
        bm = torch.from_numpy(W.boundary_mask(system)).cuda()
        X[:G.n_nodes][bm] = 0.0
    return X


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
    gen, N, m, text = WORKLOADS[args.workload]
    system = gen()
    t_setup = time.perf_counter()
    G = P.System(system)
    G.set_potential_analytic()
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    stream = torch.cuda.current_stream()
    prec = args.precision
    G.set_fp64_engine(args.fp64_engine)
    X = initial_block(torch, system, G, N)
    v0 = torch.from_numpy(W.lanczos_start(system)).cuda()
    eps_start, _ = G.rayleigh_ritz(X, residuals=False)
    # column tile of the tensor-core cell kernel for this system and N (autotuner)
    tile, tile_ms = G.autotune(N, prec) if prec in ("tf32", "tf32x3") else (None, None)
    # the start of every leg, kept in pinned host memory (also the e2e input)
    X_host = torch.empty(X.shape, dtype=X.dtype, pin_memory=True)
    X_host.copy_(X)
    flops_step = filter_flops(G.n_cells, G.n_coupling, G.n_enrich, N, m)

    def one_step(Xb, eps_prev, p):
        b = G.upper_bound(v0, 10)
        G.chfsi_step(Xb, m, eps_prev.max(), b, eps_prev.min(), precision=p,
                     fp64_tail=(args.fp64_tail if p != "fp64" else 0))
        e, _ = G.rayleigh_ritz(Xb, residuals=False)
        return e

    def timed(p, warm, steps, engine, timing=False):
        G.set_fp64_engine(engine)
        X.copy_(X_host)
        e = eps_start.copy()
        for _ in range(warm):
            e = one_step(X, e, p)
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
            e = one_step(X, e, p)
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
        return ms, e, launches // max(steps, 1), clocks, stats

    ms, eps_m, launches, clocks, stats = timed(prec, args.warmup, args.steps, args.fp64_engine, timing=True)
    # residuals of the final Ritz pairs (one more Rayleigh-Ritz, untimed)
    _, res_m = G.rayleigh_ritz(X, residuals=True)
    value = world * flops_step / (ms * 1e-3) / 1e12
    # the two tensor-core kernels of the step: the mixed filter's cell products and the
    # FP64 engine (tail degrees, Cholesky-QR, Rayleigh-Ritz); the roofline object
    # describes the one with the larger share of the step time, the other sits beside it
    (n_launch, k_ms, cellcols), (oz_launch, oz_ms, oz_flops) = stats
    s_el = {"fp64": 8, "fp32": 4, "tf32": 4, "tf32x3": 4, "bf16": 2}[prec]
    # algorithmic bytes of one cell product of N columns: the cell matrix plus
    # the 64 unique nodes' rows read (Y) and written (W)
    per_cell_bytes = NL * NL * s_el + 2.0 * 64 * N * s_el
    alg_bytes = per_cell_bytes * cellcols / float(N)
    alg_flops = 2.0 * NL * NL * cellcols
    hbm_peak, peak_src = peaks()
    cells_per_launch = cellcols / float(max(n_launch, 1) * N)
    if prec in ("fp32", "fp64"):
        # SIMT-bound: FP32 FFMA peak from 152 SMs x 128 lanes x 2 flop x 2.07 GHz; FP64 from the nominal rate
        peak = 80.5 if prec == "fp32" else 1.25
        achieved = alg_flops / (k_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": f"k_cell_apply<{'float' if prec == 'fp32' else 'double'}>",
                "launches": n_launch, "avg_launch_ms": k_ms / max(n_launch, 1),
                "peak_source": "derived from unit counts and max clock" if prec == "fp32" else "nominal FP64"}
    else:
        achieved = alg_bytes / (k_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                "traffic": None, "algorithmic_bytes_per_launch": alg_bytes / max(n_launch, 1),
                "algorithmic_bytes_per_cell": per_cell_bytes, "cells_per_launch": cells_per_launch,
                "kernel": "k_cell_tc3<%s>" % ("true" if prec == "tf32x3" else "false"),
                "launches": n_launch, "algorithmic_tflops": alg_flops / (k_ms * 1e-3) / 1e12,
                "avg_launch_ms": k_ms / max(n_launch, 1), "peak_source": peak_src}
    roof_oz = None
    if oz_launch > 0 and oz_ms > 0:
        bf16_peak, bf16_src = peaks_bf16()
        oz_tf = oz_flops / (oz_ms * 1e-3) / 1e12
        roof_oz = {"bound": "tensor", "achieved": 28.0 * oz_tf, "peak": bf16_peak, "unit": "TFLOP/s",
                   "frac": 28.0 * oz_tf / bf16_peak, "traffic": None,
                   "kernel": "k_oz (FP64-grade products)", "launches": oz_launch, "avg_launch_ms": oz_ms / oz_launch,
                   "fp64_grade_tflops": oz_tf, "algorithmic_fp64_flops_per_launch": oz_flops / oz_launch,
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
            "config": {"workload": text, "nodes": G.n_nodes, "cells": G.n_cells, "n_enrich": G.n_enrich,
                       "n_coupling": G.n_coupling, "n_qpoints": G.n_qpoints, "N": N, "m": m,
                       "fp64_tail": args.fp64_tail if prec != "fp64" else 0, "fp64_engine": args.fp64_engine,
                       "l2": "vector blocks and cell matrices exceed the 129 MB L2 (no flush needed)",
                       "step": "Lanczos bound (10) + degree-m filter + CholQR + Rayleigh-Ritz (Ritz values)",
                       "filter_flops_per_step": flops_step, "setup_s": t_setup,
                       "cell_tile": tile, "cell_tile_ms": None if tile_ms is None else [float(x) for x in tile_ms]},
            "s_per_step": ms * 1e-3, "gpu_launches": launches, "roofline": roof}
    if roof_other is not None:
        line["roofline_other_kernel"] = roof_other
    line["kernel_ms_per_step"] = {"k_cell_tc3": k_ms / args.steps, "k_oz": oz_ms / args.steps}
    line["shifted_cholqr_passes_total"] = G.rr_shifted_passes()
    if clocks:
        line["clocks"] = clocks
    line["eigs_head"] = [float(x) for x in eps_m[:5]]
    line["max_resid"] = float(res_m.max())
    # FP64 mode of the same step (from the same start)
    if not args.no_fp64 and prec != "fp64" and args.fp64_steps > 0:
        leg = {}
        engines = ["tensor"] if args.workload == "si280" else ["dfma", "tensor"]
        for eng in engines:
            ms64, eps64, _, _, _ = timed("fp64", 0, args.fp64_steps, eng)
            leg[eng] = (ms64, eps64)
        _, eps_chk, _, _, _ = timed(prec, 0, args.fp64_steps, args.fp64_engine)
        ref_eng = "dfma" if "dfma" in leg else "tensor"
        ms64, eps64 = leg[ref_eng]
        line["fp64"] = {"ms_per_step": ms64, "tflops": flops_step / (ms64 * 1e-3) / 1e12,
                        "engine": {"dfma": "dfma (plain FP64)",
                                   "tensor": "FP64-grade products on the BF16 tensor cores (cell, Gram, rotation and dense products); FP64-grade double-float enrichment coupling on the FP32 pipe"}
                        [ref_eng],
                        "speedup_mixed_vs_fp64": ms64 / ms,
                        "max_abs_eig_diff_vs_fp64_Ha": float(np.abs(eps_chk - eps64).max()),
                        "steps_compared": args.fp64_steps,
                        "from": "the same Rayleigh-Ritz-rotated start block for both modes"}
        if "dfma" in leg and "tensor" in leg:
            line["fp64_tensor_engine"] = {"ms_per_step": leg["tensor"][0],
                                          "tflops": flops_step / (leg["tensor"][0] * 1e-3) / 1e12,
                                          "max_abs_eig_diff_vs_dfma_Ha":
                                              float(np.abs(leg["tensor"][1] - leg["dfma"][1]).max())}
    # end to end through the public API with host buffers: every step copies X in
    # from pinned host memory and the filtered, rotated X back out
    if not args.no_e2e:
        G.set_fp64_engine(args.fp64_engine)
        e = eps_start.copy()
        n_e2e = 1 if args.workload == "si280" else args.steps
        X_out = torch.empty(X.shape, dtype=X.dtype, pin_memory=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            X.copy_(X_host, non_blocking=True)
            e = one_step(X, e, prec)
            X_out.copy_(X, non_blocking=True)
        torch.cuda.synchronize()
        te = (time.perf_counter() - t0) / n_e2e
        nb = X.numel() * 8
        line["e2e"] = {"value": world * flops_step / te / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": nb,
                       "d2h_bytes_per_step": nb + 8 * N, "ms_per_step": te * 1e3, "steps": n_e2e}
        del X_out
    # full SCF iterations (Sec. V) on the same system: V_eff from rho_in (Hartree
    # solve + LDA), bound, filter pass, Rayleigh-Ritz, occupations, density,
    # Hartree of rho_out, energies, Anderson mixing
    if not args.no_scf:
        G.set_fp64_engine(args.fp64_engine)
        X.copy_(X_host)
        ne = float(np.sum(system["Z"]))
        occ0, _ = P._lib.fermi(eps_start, ne, 500 * P._lib.KB_HA_PER_K)
        rho_in = G.density(X, occ0, precision="fp32" if prec != "fp64" else "fp64")
        w = G.qpoints()[:, 3]
        rho_in *= ne / float((w * rho_in).sum())
        del w
        rho_out = torch.empty_like(rho_in)
        G.scf_init(ne)
        tail = args.fp64_tail if prec != "fp64" else 0
        r0 = G.scf_step(X, rho_in, rho_out, m, precision=prec, fp64_tail=tail)   # warm-up
        torch.cuda.synchronize()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        hist = []
        for _ in range(args.scf_steps):
            hist.append(G.scf_step(X, rho_in, rho_out, m, precision=prec, fp64_tail=tail))
        s1.record(stream)
        torch.cuda.synchronize()
        ms_scf = s0.elapsed_time(s1) / max(args.scf_steps, 1)
        line["scf"] = {"s_per_iteration": ms_scf * 1e-3, "iterations_timed": args.scf_steps,
                       "n_electrons": ne, "kT_K": 500.0, "anderson_stages": 5, "mixing": 0.5,
                       "filter": f"one degree-{m} pass, {prec}", "n_qpoints": G.n_qpoints,
                       "poisson_correction_steps": [h["poisson_steps"] for h in hist],
                       "total_energy_Ha": [h["total"] for h in [r0] + hist],
                       "drho": [h["drho"] for h in [r0] + hist],
                       "start": "density of the Rayleigh-Ritz-rotated start block, renormalised to N_e"}
        del rho_in, rho_out
    # time to a converged SCF, plain FP64 against the mixed mode (small multi-atom system)
    if args.converged != "none" and rank == 0:
        line["converged_scf"] = converged_scf_section(P, torch, prec, args.converged)
    if args.dof_degree and rank == 0:
        line["dof_degree"] = dof_degree_section(P, torch)
    if args.heavy_z and rank == 0:
        line["heavy_z"] = heavy_z_section(P, torch, prec)
    # many small systems (1-6 atoms, Z in {1, 6, 8, 14}, own graded meshes, N = ceil(0.6 N_e) + 8):
    # one ChFSI filter step of every system as one CUDA graph vs the same steps launched
    # one system after another; column tiles of the cell kernel picked by the autotuner
    if args.batch and rank == 0:
        line["batch"] = batch_section(P, torch, stream)
    if not args.no_cpu and rank == 0 and world == 1:
        v, dt, desc = cpu_sample(system, N)
        line["cpu_baseline"] = {"value": v, "unit": "TFLOP/s", "cores": len(os.sched_getaffinity(0)),
                                "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
