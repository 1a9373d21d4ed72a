#!/usr/bin/env python
"""Helmholtz solves/s of HPS-preconditioned FGMRES on one GB300.

Workload (one step): the 64x64-element, N = 16 GLL, kappa = 100 scattering
problem with one seeded Gaussian bump and 16 plane-wave right-hand sides:
coefficient upload, all 4096 leaf ItI maps, 10 levels of exact merges, and
flexible GMRES (restart 60, zero initial guess) preconditioned by the merge-tree
V-cycle with 5 coarse GMRES steps, to relative residual 1e-10 per right-hand
side.  A "solve" is one right-hand side reaching that residual.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
  python bench.py --impl reference ...      (the CPU oracle, bounded sample)

Prints one JSON line (rank 0).  Under torchrun each rank solves its own seeded
problem (independent replicas, weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "64x64 elements, N=16 GLL, kappa=100, 1 seeded bump, 16 plane-wave RHS, L_exact=10, 5 coarse GMRES steps"
FP64_PEAK_NOMINAL = 1.25e12  # GB300 FP64 (nominal, vector = tensor rate)
FP32_PEAK_NOMINAL = 152 * 128 * 2 * 2.07e9  # 152 SMs x 128 FP32 lanes x FMA x 2.07 GHz
# dram read + write bytes of one leaf_ir_kernel launch at 64x64, N=16 from the committed ncu capture
# (profiles/leaf_ir_kernel_64x64_N16.md); None until captured and whenever leaf.cu changes.
LEAF_TRAFFIC_BYTES = 225.0e6  # ncu: dram read + write of one leaf_ir_kernel launch, 64x64, N=16


def _finite_or_none(x: float):
    return x if np.isfinite(x) else None


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "fallback": True}


# ---------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        for r in rows:
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), r[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


# ---------------------------------------------------------------------------- FLOP models
def leaf_flops(N: int, residuals: int = 2) -> float:
    """Executed FP32-pipe flops of the leaf kernel per element (an FMA counts 2).

    FP32 arithmetic: L D L^T of the n_i x n_i interior block (n_i^3/6 FMAs) and residuals + 1
    pairs of triangular solves with 4q right-hand sides (n_i^2 * 4q FMAs each).  Double-float
    arithmetic (pairs of FP32) counted as the FP32 operations it executes: one real product
    accumulated by the error-free dot2 is 1 MUL + 3 FMA + 8 ADD = 15 flops, a normalisation 6:
    `residuals` Kronecker-structured residuals (n_i * 4q outputs of 2q + 3 products and two
    normalisations), A = Dn_GG - Dn_Gi Z ((4q)^2 q products) and the complex Gauss-Jordan
    inverse of P ((4q)^3 complex multiply-subtracts of 4 products and 2 normalisations)."""
    q = N - 1
    ni, nb = q * q, 4 * q
    fp32 = 2.0 * (ni ** 3 / 6.0 + (residuals + 1) * ni * ni * nb)
    df = residuals * ni * nb * ((2 * q + 3) * 15 + 12) + nb * nb * q * 15 + nb ** 3 * (4 * 15 + 2 * 6)
    return fp32 + df


def leaf_flops_paper(N: int) -> float:
    """Paper-literal dense complex LU of the (N+1)^2-4 node element matrix with 4q right-hand sides."""
    nL, nG = (N + 1) ** 2 - 4, 4 * (N - 1)
    return 8.0 * (nL ** 3 / 3.0 + nL ** 2 * nG)


def matvec_flops(E: int, N: int, nrhs: int) -> float:
    nb = 4 * (N - 1)
    return 8.0 * E * nb * nb * nrhs


def matvec_bytes(E: int, N: int, nrhs: int) -> float:
    nb = 4 * (N - 1)
    return 16.0 * E * nb * nb + 3 * 16.0 * E * nb * nrhs


# ---------------------------------------------------------------------------- GPU arm
def run_gpu(args, rank, world, local_rank, dist):
    import torch

    from paper_2511_00735_gb300 import hps as H
    from paper_2511_00735_gb300 import inputs
    from paper_2511_00735_gb300 import replicas as RP

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    prob = inputs.fp64_64x64(seed=RP.seed_for_rank(rank), nrhs=args.nrhs)
    prec = H.HPS_MIXED if args.precision == "mixed" else H.HPS_FP64
    s = H.Solver(local_rank)
    s.set_outer_arith({"default": H.OUTER_DEFAULT, "fp64": H.OUTER_FP64, "df64": H.OUTER_DF64}[args.outer])
    t_host = H.setup(s, prob, prec, build=False)
    X, Y = s.node_coords()
    b_host = np.ascontiguousarray(inputs.eval_b(prob.bumps, X, Y))
    b_dev = torch.from_numpy(b_host).to(dev)
    t_dev = torch.from_numpy(t_host).to(dev)
    g_dev = torch.empty((prob.nrhs, s.n_skel), dtype=torch.complex128, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(precision, b, t, out):
        s.set_coeff(prob.kappa, b, prob.eta)
        s.build_leaves(precision)
        s.merge_levels(prob.L_exact)
        _, info = s.gmres_solve(t, tol=args.tol, inner_iters=prob.inner_iters, restart=60, max_outer=20, out=out)
        return info

    def timed(fn, k):
        # barrier + synchronize on both sides, CUDA events on the launching stream, max over ranks
        return RP.timed(fn, k, RP.CudaEventClock(stream), dist=dist, sync=lambda: torch.cuda.synchronize(dev),
                        device=dev)

    for _ in range(args.warmup):
        step(prec, b_dev, t_dev, g_dev)
    # ---- device-resident timed region ----
    clocks = ClockSampler(local_rank)
    clocks.start()
    l0 = H.kernel_launches()
    s.profile(True)
    ms, wall_ms, infos = timed(lambda: step(prec, b_dev, t_dev, g_dev), args.steps)
    prof = s.profile_read()
    s.profile(False)
    launches = H.kernel_launches() - l0
    clk = clocks.stop()
    nrhs = prob.nrhs
    value = RP.job_throughput(nrhs, args.steps, world, ms)
    its = max(i["outer_iterations"] for i in infos)
    res = max(i["max_rel_residual"] for i in infos)
    conv = min(i["converged"] for i in infos)

    # ---- end to end through the public API with host buffers ----
    g_host = np.empty((nrhs, s.n_skel), dtype=np.complex128)
    step(prec, b_host, t_host, g_host)
    e2e_ms, e2e_wall, _ = timed(lambda: step(prec, b_host, t_host, g_host), args.steps)
    h2d = b_host.nbytes + t_host.nbytes
    d2h = g_host.nbytes

    # ---- warm: cached tree, solve phase only ----
    s.set_coeff(prob.kappa, b_dev, prob.eta)
    s.build_leaves(prec)
    s.merge_levels(prob.L_exact)
    s.gmres_solve(t_dev, tol=args.tol, inner_iters=prob.inner_iters, out=g_dev)
    warm_ms, _, _ = timed(lambda: s.gmres_solve(t_dev, tol=args.tol, inner_iters=prob.inner_iters, out=g_dev),
                          args.steps)

    # ---- the plain FP64 GPU path on the same workload (comparison) ----
    fp64 = None
    if prec == H.HPS_MIXED and not args.no_fp64:
        g_mixed = g_dev.clone()  # the mixed solution of this problem (the warm solve above)
        s.set_outer_arith(H.OUTER_DEFAULT)
        step(H.HPS_FP64, b_dev, t_dev, g_dev)
        k64 = max(1, min(args.steps, 2))
        ms64, _, inf64 = timed(lambda: step(H.HPS_FP64, b_dev, t_dev, g_dev), k64)
        # the mixed result against the FP64 path's (itself the oracle's to 1e-10 in the parity tests)
        diff = torch.linalg.vector_norm(g_mixed - g_dev, dim=1) / torch.linalg.vector_norm(g_dev, dim=1)
        fp64 = {"value": k64 * nrhs * world / (ms64 / 1e3), "ms_per_step": ms64 / k64,
                "iterations": max(i["outer_iterations"] for i in inf64),
                "max_rel_residual": max(i["max_rel_residual"] for i in inf64),
                "mixed_vs_fp64_max_rel_l2": _finite_or_none(float(diff.max().item()))}
    s.close()
    return dict(outer=args.outer if args.outer != "default" else ("df64" if prec == H.HPS_MIXED else "fp64"),
                prob=prob, ms=ms, wall_ms=wall_ms, value=value, its=its, res=res, conv=conv, prof=prof,
                launches=launches, clk=clk, e2e_ms=e2e_ms, e2e_wall=e2e_wall, h2d=h2d, d2h=d2h,
                warm_ms=warm_ms, fp64=fp64)


# ---------------------------------------------------------------------------- CPU oracle
ORACLE_ITERATIONS_DEFAULT = 40  # FGMRES iterations this workload needs (same method on both sides)


def oracle_estimate(prob, iterations: int, leaf_sample: int = 48):
    """Time the CPU oracle on a bounded sample of the workload and scale to one step.

    Phases timed: `leaf_sample` leaf ItI maps (scaled to all elements); one pair
    merge per level 1..L_exact on children of the true sizes (scaled by the pairs
    per level); one FP64 skeleton matvec and one V-cycle's per-pair sweep
    operations plus the coarse GMRES steps for one right-hand side (scaled by the
    FGMRES iteration count and the number of right-hand sides)."""
    from oracle.hps import Sub, merge_pair
    from oracle.krylov import gmres_fixed
    from oracle.leaf import leaf_itI
    from oracle.problem import coefficient
    from oracle.skeleton import Mesh, apply_M

    mesh = Mesh(prob.nx, prob.nx, prob.N)
    c = coefficient(mesh, prob.kappa, prob.bumps)
    rng = np.random.default_rng(0)
    t0 = time.perf_counter()
    els = rng.choice(mesh.E, leaf_sample, replace=False)
    Ts = {}
    for e in els:
        Ts[int(e)] = leaf_itI(prob.N, mesh.h, c[e], prob.eta)["T"]
    t_leaf = (time.perf_counter() - t0) / leaf_sample * mesh.E
    # merges and the per-pair sweep work, level by level
    t_merge = 0.0
    t_sweep = 0.0
    q = mesh.q
    a, b = 1, 1
    sample_T = next(iter(Ts.values()))
    for lev in range(1, prob.L_exact + 1):
        d = "x" if lev % 2 == 1 else "y"
        s1 = Sub(mesh, 0, 0, a, b)
        s2 = Sub(mesh, a if d == "x" else 0, b if d == "y" else 0, a, b)
        for s in (s1, s2):
            if s.n == sample_T.shape[0]:
                s.T = sample_T
            else:
                Z = rng.standard_normal((s.n, s.n)) + 1j * rng.standard_normal((s.n, s.n))
                s.T = 0.5 * Z / np.sqrt(s.n)
        t1 = time.perf_counter()
        _, rec = merge_pair(mesh, s1, s2, d)
        t2 = time.perf_counter()
        npairs = mesh.E // (2 ** lev)
        t_merge += (t2 - t1) * npairs
        r = rng.standard_normal(2 * rec.m) + 0j
        y = rng.standard_normal(len(rec.y_inn)) + 0j
        t3 = time.perf_counter()
        z = rec.solveA(r)
        _ = rec.C @ z
        _ = z - rec.solveA(rec.B @ y)
        t_sweep += (time.perf_counter() - t3) * npairs
        if d == "x":
            a *= 2
        else:
            b *= 2
    # coarse GMRES on the coarse subdomains (4 blocks of a x b elements)
    nsub = mesh.E // (a * b)
    nc = 2 * (a + b) * q
    Tc = [0.5 * (rng.standard_normal((nc, nc)) + 1j * rng.standard_normal((nc, nc))) / np.sqrt(nc)
          for _ in range(min(nsub, 4))]
    v = rng.standard_normal(nc) + 0j
    t4 = time.perf_counter()
    gmres_fixed(lambda x: x + Tc[0] @ x, v, prob.inner_iters)
    t_coarse = (time.perf_counter() - t4) * nsub
    # one FP64 skeleton matvec (one right-hand side); every element uses a sampled map
    Tall = [Ts[int(els[e % leaf_sample])] for e in range(mesh.E)]
    g = rng.standard_normal(mesh.n_skel) + 0j
    t5 = time.perf_counter()
    apply_M(mesh, Tall, g)
    t_mv = time.perf_counter() - t5
    per_rhs = iterations * (t_mv + t_sweep + t_coarse)
    total = t_leaf + t_merge + prob.nrhs * per_rhs
    cores = blas_threads()
    return {"seconds_per_step": total, "t_leaf": t_leaf, "t_merge": t_merge, "t_solve_per_rhs": per_rhs,
            "cores": cores, "measured_s": time.perf_counter() - t0}


def blas_threads() -> int:
    """Threads numpy's BLAS uses (threadpoolctl when installed, else the visible cores)."""
    try:
        import threadpoolctl

        info = threadpoolctl.threadpool_info()
        return max([p.get("num_threads", 1) for p in info] + [1])
    except ImportError:
        return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def cpu_baseline_entry(prob, iterations):
    est = oracle_estimate(prob, iterations)
    return {"value": prob.nrhs / est["seconds_per_step"], "unit": "solves/s", "cores": est["cores"],
            "kind": "oracle",
            "sample": (f"{48} of {prob.nx * prob.nx} leaf maps, one pair merge per level (children of the true sizes), "
                       f"one matvec + one V-cycle's pair sweeps + {prob.inner_iters} coarse GMRES steps for one RHS "
                       f"x {iterations} FGMRES iterations x {prob.nrhs} RHS; {est['measured_s']:.1f} s of CPU work"),
            "phases_s": {"leaves": est["t_leaf"], "merges": est["t_merge"],
                         "solve_per_rhs": est["t_solve_per_rhs"]}}


# ---------------------------------------------------------------------------- batching / serving
def run_table1(args, prec):
    """Memory-time trade-off of section 5 (Table 1) on the 64x64 workload: for each number of
    exactly merged levels and each count of coarse GMRES steps, the device bytes held by the
    tree (PMem), the merge time (Bt), the FGMRES iterations (It) and the solve time (St), plus
    direct HPS (exact coarse level).  Times are CUDA events on the library's stream."""
    import torch

    from paper_2511_00735_gb300 import hps as H
    from paper_2511_00735_gb300 import inputs

    prob = inputs.fp64_64x64(seed=1, nrhs=args.nrhs)
    s = H.Solver(0)
    stream = torch.cuda.current_stream(0)
    t = H.setup(s, prob, prec, build=True)
    leaf_bytes = s.bytes_held()
    t_dev = torch.from_numpy(t).to("cuda:0")
    g_dev = torch.empty((prob.nrhs, s.n_skel), dtype=torch.complex128, device="cuda:0")

    def ev_ms(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), out

    def solve(ci):
        return s.gmres_solve(t_dev, tol=args.tol, inner_iters=ci, restart=60, max_outer=20, out=g_dev,
                             raise_on_notconv=False)[1]

    rows = []
    cases = [(lx, False) for lx in range(1, s.levels, 2)] + [(s.levels - 1, True)]
    for lx, exact in cases:
        s.release_workspace()
        bt, _ = ev_ms(lambda: s.merge_levels(lx, exact_coarse=exact))
        held = s.bytes_held()
        for ci in ([0] if exact else [2, 4, 6]):
            solve(ci)  # first solve of a tree captures the V-cycle graph
            st, info = ev_ms(lambda: solve(ci))
            rows.append({"levels": lx + 1, "L_exact": lx, "coarse": "exact" if exact else f"{ci} c.i.",
                         "pmem_bytes": held - leaf_bytes, "bytes_held_tree": held, "bt_ms": bt,
                         "it": info["outer_iterations"], "converged": info["converged"], "st_ms": st,
                         "max_rel_residual": info["max_rel_residual"]})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    s.close()
    return {"metric": "memory-time trade-off (section 5, Table 1): PMem, Bt, It, St by levels and coarse steps",
            "value": None, "unit": None, "n_gpus": 1, "dtype": "f64+f32" if prec else "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD.replace("L_exact=10, 5 coarse GMRES steps", "L_exact and coarse steps swept"),
                       "precision": args.precision, "tol": args.tol, "leaf_bytes": leaf_bytes},
            "rows": rows}


def run_systems(args):
    from paper_2511_00735_gb300 import hps as H

    prec = H.HPS_MIXED if args.precision == "mixed" else H.HPS_FP64
    clocks = ClockSampler(0)
    l0 = None
    if args.workload == "table1":
        clocks.start()
        l0 = H.kernel_launches()
        line = run_table1(args, prec)
    elif args.workload == "batch":
        from paper_2511_00735_gb300 import batch as B

        count = args.count or 512
        B.run_mix(min(count, 16), seed=99, slots=args.slots, precision=prec)  # warm-up (other seeds)
        clocks.start()
        l0 = H.kernel_launches()
        r = B.run_mix(count, seed=3, slots=args.slots, precision=prec)
        line = {"metric": "Helmholtz solves/s at rel-residual 1e-10, batching mix", "value": r["solves_per_s"],
                "unit": "solves/s", "n_gpus": 1, "higher_is_better": True, "dtype": "f64+f32" if prec else "f64",
                "data": "synthetic",
                "config": {"workload": f"{count} problems: grids U{{8,16,32,64}}^2, N U{{8,12,16}}, kappa U[20,150], "
                                       "1 bump, 1-8 RHS", "slots": args.slots, "precision": args.precision},
                **r}
    else:
        from paper_2511_00735_gb300 import serve as S

        count = args.count or 200
        reqs = S.poisson_stream(count, args.rate)
        srv = S.Server(0, workers=args.slots, precision=prec, hbm_cap=150e9)
        clocks.start()
        l0 = H.kernel_launches()
        r = S.run_stream(reqs, srv, timeout=args.serve_timeout,
                         progress=lambda m: print(m, file=sys.stderr, flush=True))
        srv.close()
        line = {"metric": "Helmholtz solves/s and p50/p99 latency at rel-residual 1e-10, serving stream",
                "value": r["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "higher_is_better": True,
                "dtype": "f64+f32" if prec else "f64", "data": "synthetic",
                "config": {"workload": f"{count} Poisson arrivals at {args.rate}/s: 90% batching-mix trees, "
                                       "10% 128x128 N=16 kappa=200 trees, 1-64 RHS per request, 150 GB cap",
                           "workers": args.slots, "precision": args.precision},
                **r}
    line["gpu_launches"] = H.kernel_launches() - l0
    line["clocks"] = clocks.stop()
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--nrhs", type=int, default=16)
    ap.add_argument("--outer", default="default", choices=["default", "fp64", "df64"],
                    help="outer FGMRES arithmetic (default: df64 for mixed, fp64 for fp64)")
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison run")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--workload", default="scattering64", choices=["scattering64", "batch", "serve", "table1"],
                    help="scattering64: the timed step above; batch: the 512-problem mix; serve: a Poisson stream; "
                         "table1: the memory-time trade-off over exact levels and coarse steps")
    ap.add_argument("--count", type=int, default=0, help="problems (batch) or requests (serve)")
    ap.add_argument("--rate", type=float, default=200.0, help="serve: arrivals per second")
    ap.add_argument("--slots", type=int, default=8, help="batch slots / serve workers")
    ap.add_argument("--serve-timeout", type=float, default=240.0, help="serve: stop waiting after this many seconds")
    args = ap.parse_args()
    if args.workload != "scattering64":
        return run_systems(args)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    from paper_2511_00735_gb300 import inputs

    if args.impl == "reference":
        if rank != 0:
            return
        prob = inputs.fp64_64x64(seed=1, nrhs=args.nrhs)
        vals = []
        for i in range(args.warmup + args.steps):
            est = oracle_estimate(prob, ORACLE_ITERATIONS_DEFAULT, leaf_sample=16)
            if i >= args.warmup:
                vals.append(prob.nrhs / est["seconds_per_step"])
        v = statistics.median(vals)
        line = {"metric": "Helmholtz solves/s at rel-residual 1e-10", "value": v, "unit": "solves/s",
                "impl": "reference", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * prob.nrhs / v, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "global_batch": prob.nrhs, "parallelism": "replicas"},
                "cpu_baseline": {"value": v, "unit": "solves/s", "kind": "oracle", "cores": est["cores"],
                                 "sample": f"16 leaf maps, one merge per level, one V-cycle's pair sweeps, one matvec "
                                           f"(one RHS) scaled by {ORACLE_ITERATIONS_DEFAULT} iterations x "
                                           f"{prob.nrhs} RHS"},
                "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    dist = None
    if world > 1:
        import torch.distributed as tdist

        tdist.init_process_group("nccl")
        dist = tdist
    r = run_gpu(args, rank, world, local_rank, dist)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    prob = r["prob"]
    peaks = load_peaks()
    nrhs = prob.nrhs
    prof = r["prof"]
    E, N = prob.nx * prob.nx, prob.N
    # dominant single-kernel phase: the leaf build (one launch per step) or the FP64 matvec (one launch per call)
    leaf_ms, leaf_launch, leaf_calls = prof["leaf"]
    mv_ms, mv_launch, mv_calls = prof["matvec"]
    cand = []
    if leaf_calls:
        per = leaf_ms / leaf_calls
        f32 = leaf_flops(N) * E
        lit = leaf_flops_paper(N) * E
        cand.append((leaf_ms, {"kernel": "leaf_ir_kernel (leaf ItI maps: FP32 factor, double-float refinement "
                                         "and inverse)",
                               "bound": "alu", "achieved": f32 / (per / 1e3) / 1e12,
                               "peak": FP32_PEAK_NOMINAL / 1e12, "unit": "TFLOP/s",
                               "frac": f32 / (per / 1e3) / FP32_PEAK_NOMINAL,
                               "traffic": LEAF_TRAFFIC_BYTES if prob.nx == 64 and N == 16 else None,
                               "traffic_unit": "bytes per launch (ncu dram read + write)",
                               "flops_per_launch": f32, "ms_per_launch": per,
                               "paper_literal_flops_per_launch": lit,
                               "paper_literal_rate_tflops": lit / (per / 1e3) / 1e12,
                               "peak_source": "FP32 pipes from unit counts and clock: 152 SMs x 128 lanes x "
                                              "2 (FMA) x 2.07 GHz = 80.5 TFLOP/s (double-float counted as the "
                                              "FP32 operations it executes)"}))
    if mv_calls and r.get("outer") == "fp64":
        per = mv_ms / mv_calls
        fl = matvec_flops(E, N, nrhs)
        cand.append((mv_ms, {"kernel": "es_matvec_kernel (skeleton matvec, FP64)", "bound": "alu",
                             "achieved": fl / (per / 1e3) / 1e12, "peak": FP64_PEAK_NOMINAL / 1e12,
                             "unit": "TFLOP/s", "frac": fl / (per / 1e3) / FP64_PEAK_NOMINAL,
                             "traffic": None, "flops_per_launch": fl, "ms_per_launch": per,
                             "peak_source": "nominal GB300 FP64 (1.25 TFLOP/s)"}))
    roof = max(cand, key=lambda x: x[0])[1] if cand else None
    cpu = None
    if not args.no_cpu and world == 1:
        cpu = cpu_baseline_entry(prob, r["its"])
    line = {
        "metric": "Helmholtz solves/s at rel-residual 1e-10 (mixed vs FP64)",
        "value": r["value"], "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": r["ms"] / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64+f32" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "global_batch": nrhs * world, "precision": args.precision,
                   "outer": args.outer if args.outer != "default" else ("df64" if args.precision == "mixed" else "fp64"),
                   "tol": args.tol, "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2: leaf maps 236 MB, merge tree ~1.3 GB, Krylov basis 3.8 GB per step"},
        "iterations": r["its"], "max_rel_residual": r["res"], "converged": r["conv"],
        "e2e": {"value": args.steps * nrhs * world / (r["e2e_ms"] / 1e3), "unit": "solves/s",
                "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"],
                "wall_value": args.steps * nrhs * world / (r["e2e_wall"] / 1e3)},
        "warm": {"value": args.steps * nrhs * world / (r["warm_ms"] / 1e3), "unit": "solves/s",
                 "note": "cached leaf maps and merge tree, solve phase only"},
        "fp64": r["fp64"],
        "gpu_launches": r["launches"],
        "phases_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "launches_per_step": {k: v[1] / args.steps for k, v in prof.items()},
        "roofline": roof,
        "cpu_baseline": cpu,
        "clocks": r["clk"],
        "peaks": {"hbm_gbs": peaks.get("hbm_gbs"), "bf16_tflops": peaks.get("bf16_tflops"),
                  "fp64_tflops_nominal": FP64_PEAK_NOMINAL / 1e12},
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
