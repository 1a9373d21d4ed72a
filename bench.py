#!/usr/bin/env python
"""Helmholtz solves/s (and per-step p50/p99 latency) of HPS-preconditioned FGMRES on one GB300.

Workload (one step, default): the 128x128-element, N = 16 GLL, kappa = 200 scattering
problem with eight seeded Gaussian bumps and 32 plane-wave right-hand sides:
coefficient upload, all 16384 leaf ItI maps, 12 levels of exact merges, and
flexible GMRES (restart 20, zero initial guess) preconditioned by the merge-tree
V-cycle with 5 coarse GMRES steps, to an FP64 relative residual of 1e-10 per
right-hand side.  A "solve" is one right-hand side whose returned solution has
that FP64 residual; only those are counted.  The plain FP64 path is timed on the
same problem and the mixed solution's difference from it is stated.  The restart length
is a memory/time trade-off of the same method (Table 1 of the paper used 60 to bound a
laptop's memory): each restart costs one FP64 residual, each Arnoldi step j a Gram-Schmidt
pass over j basis vectors; --restart 60 reproduces that setting, and the line carries the
warm solve at restart 60 beside the headline.
--workload scattering64 runs the 64x64, N = 16, kappa = 100 problem (16 RHS).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
  python bench.py --impl reference ...      (the CPU oracle, bounded sample)
  python bench.py --workload batch|serve|table1|phase ...

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

# the headline metric, the same string in both arms
METRIC = "Helmholtz solves/s & p50/p99 latency at rel-residual 1e-10, mixed vs FP64"
WORKLOADS = {
    "scattering128": ("128x128 elements, N=16 GLL, kappa=200, 8 seeded bumps, 32 plane-wave RHS, L_exact=12, "
                      "5 coarse GMRES steps", 32, 2),
    "scattering64": ("64x64 elements, N=16 GLL, kappa=100, 1 seeded bump, 16 plane-wave RHS, L_exact=10, "
                     "5 coarse GMRES steps", 16, 1),
}
FP64_PEAK_NOMINAL = 1.25e12  # GB300 FP64 (nominal, vector = tensor rate)
FP32_PEAK_NOMINAL = 152 * 128 * 2 * 2.07e9  # 152 SMs x 128 FP32 lanes x FMA x 2.07 GHz
# ncu dram read + write of one leaf_ir_kernel launch per element (64x64, N=16 capture, scaled by
# the elements of a launch); None whenever leaf.cu changed since the capture
LEAF_TRAFFIC_BYTES_PER_ELEMENT = (12.34e6 + 229.55e6) / 4096
# ncu dram read + write of the bf16x3 sweep kernel over one V-cycle's launches divided by their
# algorithmic bytes (64x64, N=16, 32 RHS capture: the ratio scales the full-size launches);
# None until captured, and whenever tc.cu's sweep kernel changed since
SWEEP_TRAFFIC_RATIO = 1748.66e6 / 1893.34e6
TF32_OVER_BF16 = 1.1 / 2.25  # nominal dense tensor rates: tf32 / bf16
KPROF_APPLIES = 8  # preconditioner applications of the per-kernel timing pass


def make_problem(workload: str, seed: int, nrhs: int):
    from paper_2511_00735_gb300 import inputs

    if workload == "scattering128":
        return inputs.mixed_128x128(seed=seed, nrhs=nrhs)
    return inputs.fp64_64x64(seed=seed, nrhs=nrhs)


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


# ---------------------------------------------------------------------------- V-cycle bytes
def vcycle_bytes(nx: int, N: int, L_exact: int, nrhs: int, inner_iters: int, elem: int = 8) -> dict:
    """Algorithmic HBM bytes of one V-cycle application of the FP32 tree (complex: `elem` bytes).

    Operators, each read once: per merge level l the restriction U [2p x 2m] and the
    prolongation Dm [2m x 2n] of every pair (n = a child's boundary length, m = its interface
    length, p = n - m), and per coarse GMRES step the interior-interior block of every coarse
    subdomain's map.  Block vectors: each stage's sweep vector (rows = subdomains x boundary
    length, nrhs columns) read and written once on the way up and once on the way down, plus
    the stage-0 entry gather and exit scatter (the caller's vectors read and written once)."""
    q = N - 1
    E = nx * nx
    a = b = 1
    ops = 0
    vec_rows = 4 * q * E  # stage 0
    vec = 0
    for lev in range(1, L_exact + 1):
        n = 2 * (a + b) * q
        m = (b if lev % 2 == 1 else a) * q
        p = n - m
        npairs = E >> lev
        ops += npairs * (2 * p * 2 * m + 2 * m * 2 * n)
        vec += 2 * 2 * vec_rows  # up: read stage l-1, write stage l; down: the same, reversed
        if lev % 2 == 1:
            a *= 2
        else:
            b *= 2
        vec_rows = (E >> lev) * 2 * (a + b) * q
    gx, gy = nx // a, nx // b
    coarse = 0
    for iy in range(gy):
        for ix in range(gx):
            ni = q * ((b if ix > 0 else 0) + (b if ix < gx - 1 else 0) + (a if iy > 0 else 0) + (a if iy < gy - 1 else 0))
            coarse += ni * ni
    vec += 2 * 2 * 4 * q * E  # entry gather, exit scatter
    total = elem * (ops + inner_iters * coarse) + elem * nrhs * vec
    return {"bytes": total, "operator_bytes": elem * (ops + inner_iters * coarse), "vector_bytes": elem * nrhs * vec}


# ---------------------------------------------------------------------------- GPU arm
def run_gpu(args, rank, world, local_rank, dist):
    import torch

    from paper_2511_00735_gb300 import hps as H
    from paper_2511_00735_gb300 import inputs
    from paper_2511_00735_gb300 import replicas as RP

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    _, _, base_seed = WORKLOADS[args.workload]
    prob = make_problem(args.workload, RP.seed_for_rank(rank, base=base_seed), args.nrhs)
    prec = H.HPS_MIXED if args.precision == "mixed" else H.HPS_FP64
    s = H.Solver(local_rank)
    s.set_outer_arith({"default": H.OUTER_DEFAULT, "fp64": H.OUTER_FP64, "df64": H.OUTER_DF64}[args.outer])
    pinned = []  # page-locked host buffers of the end-to-end measurement (kept alive here)

    def pin(a):
        t = torch.empty(a.shape, dtype=torch.from_numpy(a[:0]).dtype, pin_memory=True)
        pinned.append(t)
        out = t.numpy()
        out[...] = a
        return out

    t_host = pin(H.setup(s, prob, prec, build=False))
    X, Y = s.node_coords()
    b_host = pin(np.ascontiguousarray(inputs.eval_b(prob.bumps, X, Y)))
    b_dev = torch.from_numpy(b_host).to(dev)
    t_dev = torch.from_numpy(t_host).to(dev)
    g_dev = torch.empty((prob.nrhs, s.n_skel), dtype=torch.complex128, device=dev)
    stream = torch.cuda.current_stream(dev)
    s.set_autotune(H.TUNE_ON if args.autotune == "on" else H.TUNE_OFF)

    def step(precision, b, t, out):
        s.set_coeff(prob.kappa, b, prob.eta)
        s.build_leaves(precision)
        s.merge_levels(prob.L_exact)
        _, info = s.gmres_solve(t, tol=args.tol, inner_iters=prob.inner_iters, restart=args.restart,
                                max_outer=args.max_outer, out=out, raise_on_notconv=False)
        return info

    def timed(fn, k):
        # barrier + synchronize on both sides, CUDA events on the launching stream, max over ranks
        clock = RP.CudaEventClock(stream)
        ms, wall, outs = RP.timed(fn, k, clock, dist=dist, sync=lambda: torch.cuda.synchronize(dev), device=dev)
        return ms, wall, outs, clock.laps_ms()

    for _ in range(args.warmup):
        step(prec, b_dev, t_dev, g_dev)
    # ---- device-resident timed region ----
    clocks = ClockSampler(local_rank)
    clocks.start()
    l0 = H.kernel_launches()
    s.profile(True)
    ms, wall_ms, infos, laps = timed(lambda: step(prec, b_dev, t_dev, g_dev), args.steps)
    prof = s.profile_read()
    s.profile(False)
    launches = H.kernel_launches() - l0
    clk = clocks.stop()
    nrhs = prob.nrhs
    conv_total = sum(i["converged"] for i in infos)  # solves whose FP64 residual reached tol
    value = RP.sum_over_ranks(conv_total, dist, dev) / (ms / 1e3)  # all ranks' solves / slowest rank's time
    its = max(i["outer_iterations"] for i in infos)
    res = max(i["max_rel_residual"] for i in infos)
    conv = min(i["converged"] for i in infos)

    # ---- end to end through the public API with host buffers ----
    g_host = pin(np.zeros((nrhs, s.n_skel), dtype=np.complex128))
    step(prec, b_host, t_host, g_host)
    e2e_ms, e2e_wall, e2e_infos, _ = timed(lambda: step(prec, b_host, t_host, g_host), args.steps)
    e2e_conv = RP.sum_over_ranks(sum(i["converged"] for i in e2e_infos), dist, dev)
    h2d = b_host.nbytes + t_host.nbytes
    d2h = g_host.nbytes

    # ---- warm: cached tree, solve phase only ----
    s.set_coeff(prob.kappa, b_dev, prob.eta)
    s.build_leaves(prec)
    s.merge_levels(prob.L_exact)
    s.gmres_solve(t_dev, tol=args.tol, inner_iters=prob.inner_iters, restart=args.restart,
                  max_outer=args.max_outer, out=g_dev)
    warm_ms, _, warm_infos, warm_laps = timed(
        lambda: s.gmres_solve(t_dev, tol=args.tol, inner_iters=prob.inner_iters, restart=args.restart,
                              max_outer=args.max_outer, out=g_dev, raise_on_notconv=False)[1], args.steps)
    warm_conv = RP.sum_over_ranks(sum(i["converged"] for i in warm_infos), dist, dev)
    # the same warm solve at the paper's restart length (60)
    r60 = None
    if args.restart != 60:
        r60_ms, _, r60_infos, _ = timed(
            lambda: s.gmres_solve(t_dev, tol=args.tol, inner_iters=prob.inner_iters, restart=60, max_outer=20,
                                  out=g_dev, raise_on_notconv=False)[1], 1)
        r60 = {"value": RP.sum_over_ranks(r60_infos[0]["converged"], dist, dev) / (r60_ms / 1e3), "unit": "solves/s",
               "iterations": r60_infos[0]["outer_iterations"], "max_rel_residual": r60_infos[0]["max_rel_residual"],
               "note": "warm solve (cached tree) with restart 60; compare with warm"}

    # ---- per-launch timing of the sweep products and the merge GEMMs ----
    # Inside the step the V-cycle replays as one CUDA graph, whose launches cannot be bracketed
    # one by one: the same tree (rebuilt once) and KPROF_APPLIES direct applications of the same
    # V-cycle on a random block of nrhs right-hand sides, each launch of a class between CUDA
    # events on the context's stream (the stream the kernels are launched on).
    kern = None
    if prec == H.HPS_MIXED:
        s.set_coeff(prob.kappa, b_dev, prob.eta)
        s.build_leaves(prec)
        s.profile_kernels(True)
        s.merge_levels(prob.L_exact)
        gen = torch.Generator(device=dev).manual_seed(7)
        rr = torch.complex(torch.randn((nrhs, s.n_skel), generator=gen, device=dev, dtype=torch.float64),
                           torch.randn((nrhs, s.n_skel), generator=gen, device=dev, dtype=torch.float64))
        for _ in range(KPROF_APPLIES):
            s.precond_apply(rr, inner_iters=prob.inner_iters)
        kern = s.profile_kernels_read()
        s.profile_kernels(False)
        kern["applies"] = KPROF_APPLIES
        kern["precond_calls_per_step"] = prof["precond"][2] / args.steps
    tune_table = H.autotune_table() if args.autotune == "on" else ""

    # ---- the plain FP64 GPU path on the same workload (comparison) ----
    fp64 = None
    if prec == H.HPS_MIXED and not args.no_fp64:
        g_mixed = g_dev.clone()  # the mixed solution of this problem (the warm solve above)
        s.set_outer_arith(H.OUTER_DEFAULT)
        s.release_workspace()
        step(H.HPS_FP64, b_dev, t_dev, g_dev)
        ms64, _, inf64, _ = timed(lambda: step(H.HPS_FP64, b_dev, t_dev, g_dev), 1)
        # the mixed result against the FP64 path's (itself the oracle's to 1e-10 in the parity tests)
        diff = torch.linalg.vector_norm(g_mixed - g_dev, dim=1) / torch.linalg.vector_norm(g_dev, dim=1)
        fp64 = {"value": RP.sum_over_ranks(inf64[0]["converged"], dist, dev) / (ms64 / 1e3), "unit": "solves/s", "ms_per_step": ms64,
                "steps": 1, "iterations": inf64[0]["outer_iterations"],
                "max_rel_residual": inf64[0]["max_rel_residual"], "converged": inf64[0]["converged"],
                "mixed_vs_fp64_max_rel_l2": _finite_or_none(float(diff.max().item())),
                "note": "max over right-hand sides of ||g_mixed - g_fp64||_2 / ||g_fp64||_2"}
        s.release_workspace()
    s.close()
    return dict(outer=args.outer if args.outer != "default" else ("df64" if prec == H.HPS_MIXED else "fp64"),
                prob=prob, ms=ms, wall_ms=wall_ms, value=value, its=its, res=res, conv=conv, prof=prof,
                launches=launches, clk=clk, e2e_ms=e2e_ms, e2e_wall=e2e_wall, e2e_conv=e2e_conv, h2d=h2d, d2h=d2h,
                warm_ms=warm_ms, warm_conv=warm_conv, warm_laps=warm_laps, fp64=fp64, laps=laps, r60=r60,
                kern=kern, tune_table=tune_table)


# ---------------------------------------------------------------------------- CPU oracle
# FGMRES iterations of each workload's seeded problem (the same method on both sides; the GPU
# arm passes the count its own run took)
ORACLE_ITERATIONS = {"scattering128": 48, "scattering64": 40}


def _best_time(fn, min_s: float = 0.05, reps: int = 3) -> float:
    """Seconds of one call of fn: the fastest of `reps` batches, each repeated until it lasts
    `min_s` (short operations are timed many times so host timer noise does not get scaled)."""
    best = float("inf")
    for _ in range(reps):
        n, t = 0, 0.0
        t0 = time.perf_counter()
        while n == 0 or t < min_s:
            fn()
            n += 1
            t = time.perf_counter() - t0
        best = min(best, t / n)
    return best


class OracleSampler:
    """The CPU oracle as it stands, timed on bounded samples of one step of a workload and scaled
    to the whole step.

    Leaves: the 16 elements of a 4x4 block plus `leaf_sample` seeded elsewhere, timed one by one
    (median, scaled by E).  Merges: every pair merge of levels 1-4 of that block on its real maps
    (timed, scaled by the pairs of each level); from level 5 up one pair merge per level on
    children of the true sizes whose maps are drawn at random (the merge's dense LU and products
    cost the same whatever the values).  Solve, per right-hand side and FGMRES iteration: one
    FP64 skeleton matvec over all elements, one V-cycle's per-pair sweep operations (timed per
    level, scaled by its pairs) and the coarse GMRES steps; scaled by the iteration count and the
    right-hand sides."""

    def __init__(self, workload: str, nrhs: int, iterations: int):
        from oracle.skeleton import Mesh
        from paper_2511_00735_gb300 import inputs

        self.prob = make_problem(workload, WORKLOADS[workload][2], nrhs)
        self.mesh = Mesh(self.prob.nx, self.prob.nx, self.prob.N)
        self.iterations = iterations
        self.inputs = inputs
        self.big_merge_s = {}  # level -> seconds of one pair merge on random children (levels >= 9)

    def c_of(self, e: int):
        X, Y = self.mesh.node_xy(e)  # c = kappa^2 (1 - b) at the oracle's own nodes of element e
        return self.prob.kappa ** 2 * (1.0 - self.inputs.eval_b(self.prob.bumps, X, Y))

    def sample(self, seed: int, leaf_sample: int = 8) -> dict:
        from oracle.hps import Sub, merge_pair
        from oracle.krylov import gmres_fixed
        from oracle.leaf import leaf_itI
        from oracle.skeleton import apply_M

        prob, mesh = self.prob, self.mesh
        q = mesh.q
        rng = np.random.default_rng(seed)
        t_start = time.perf_counter()
        block = [mesh.elem(ix, iy) for iy in range(4) for ix in range(4)]
        others = [int(x) for x in rng.choice(mesh.E, leaf_sample, replace=False)]
        Ts, t_leaves = {}, []
        for e in block + others:
            ce = self.c_of(e)
            t0 = time.perf_counter()
            T = leaf_itI(prob.N, mesh.h, ce, prob.eta)["T"]
            t_leaves.append(time.perf_counter() - t0)
            Ts.setdefault(e, T)
        t_leaf = float(np.median(t_leaves)) * mesh.E
        subs = {}
        for e in block:
            ix, iy = e % mesh.nx, e // mesh.nx
            sb = Sub(mesh, ix, iy, 1, 1)
            sb.T = Ts[e]
            subs[(ix, iy)] = sb
        t_merge = t_sweep = 0.0
        a, b = 1, 1
        for lev in range(1, prob.L_exact + 1):
            d = "x" if lev % 2 == 1 else "y"
            npairs = mesh.E // (2 ** lev)
            if a * (2 if d == "x" else 1) <= 4 and b * (2 if d == "y" else 1) <= 4:
                pairs = [(k, (k[0] + a, k[1]) if d == "x" else (k[0], k[1] + b)) for k in subs
                         if (d == "x" and (k[0] // a) % 2 == 0) or (d == "y" and (k[1] // b) % 2 == 0)]
            elif lev in self.big_merge_s:
                # levels >= 9: the merge on random children was timed by the first (warm-up) sample;
                # its dense LU and products cost the same on every sample.  Its sweep operations are
                # still timed below, on children of the true sizes.
                t_merge += self.big_merge_s[lev] * npairs
                s1 = Sub(mesh, 0, 0, a, b)
                s2 = Sub(mesh, a if d == "x" else 0, b if d == "y" else 0, a, b)
                m = (b if d == "x" else a) * q
                n2 = 2 * (s1.n - m)
                lu = __import__("scipy.linalg", fromlist=["lu_factor"]).lu_factor(
                    np.eye(2 * m) + 0.1 * (rng.standard_normal((2 * m, 2 * m)) + 0j))
                Bm = rng.standard_normal((2 * m, n2)) + 0j
                Cm = rng.standard_normal((n2, 2 * m)) + 0j
                r = rng.standard_normal(2 * m) + 0j
                y = rng.standard_normal(n2) + 0j
                sla = __import__("scipy.linalg", fromlist=["lu_solve"])
                t_sweep += _best_time(lambda: (Cm @ sla.lu_solve(lu, r), sla.lu_solve(lu, Bm @ y)), min_s=0.01,
                                      reps=1) * npairs
                subs = {}
                if d == "x":
                    a *= 2
                else:
                    b *= 2
                continue
            else:
                s1 = Sub(mesh, 0, 0, a, b)
                s2 = Sub(mesh, a if d == "x" else 0, b if d == "y" else 0, a, b)
                for sb in (s1, s2):
                    Z = rng.standard_normal((sb.n, sb.n)) + 1j * rng.standard_normal((sb.n, sb.n))
                    sb.T = 0.5 * Z / np.sqrt(sb.n)
                subs = {(0, 0): s1, ((a, 0) if d == "x" else (0, b)): s2}
                pairs = [((0, 0), (a, 0) if d == "x" else (0, b))]
            new_subs, tm, ts = {}, 0.0, 0.0
            for k1, k2 in pairs:
                t1 = time.perf_counter()
                merged, rec = merge_pair(mesh, subs[k1], subs[k2], d)
                tm += time.perf_counter() - t1
                r = rng.standard_normal(2 * rec.m) + 0j
                y = rng.standard_normal(len(rec.y_inn)) + 0j
                ts += _best_time(lambda: (rec.C @ rec.solveA(r), rec.solveA(rec.B @ y)), min_s=0.01, reps=1)
                new_subs[k1] = merged
            t_merge += tm / len(pairs) * npairs
            t_sweep += ts / len(pairs) * npairs
            if lev >= 9:
                self.big_merge_s[lev] = tm / len(pairs)
            subs = new_subs
            if d == "x":
                a *= 2
            else:
                b *= 2
        nsub = mesh.E // (a * b)
        nc = 2 * (a + b) * q
        Tc = 0.5 * (rng.standard_normal((nc, nc)) + 1j * rng.standard_normal((nc, nc))) / np.sqrt(nc)
        v = rng.standard_normal(nc) + 0j
        t_coarse = _best_time(lambda: gmres_fixed(lambda x: x + Tc @ x, v, prob.inner_iters), min_s=0.02,
                              reps=1) * nsub
        keys = list(Ts)
        Tall = [Ts[keys[e % len(keys)]] for e in range(mesh.E)]
        g = rng.standard_normal(mesh.n_skel) + 0j
        t_mv = _best_time(lambda: apply_M(mesh, Tall, g), min_s=0.0, reps=1)
        per_rhs = self.iterations * (t_mv + t_sweep + t_coarse)
        total = t_leaf + t_merge + prob.nrhs * per_rhs
        return {"seconds_per_step": total, "solves_per_s": prob.nrhs / total, "t_leaf": t_leaf,
                "t_merge": t_merge, "t_solve_per_rhs": per_rhs, "measured_s": time.perf_counter() - t_start,
                "leaf_sample": len(t_leaves)}


def oracle_samples(workload: str, nrhs: int, iterations: int, samples: int) -> dict:
    """One warm-up sample and `samples` timed ones of the oracle (seeds 1..samples)."""
    smp = OracleSampler(workload, nrhs, iterations)
    smp.sample(0)
    runs = [smp.sample(k + 1) for k in range(samples)]
    return {"runs": runs, "nrhs": smp.prob.nrhs}


def _oracle_subprocess(workload: str, nrhs: int, iterations: int, threads: int, samples: int) -> dict:
    """oracle_samples in a fresh interpreter whose BLAS and OpenMP pools have `threads` threads
    (set before numpy loads), so the timing does not depend on what this process imported."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = str(threads)
    env["CUDA_VISIBLE_DEVICES"] = ""
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", workload, "--nrhs", str(nrhs),
           "--oracle-iterations", str(iterations), "--steps", str(samples)]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(f"oracle sample failed: {r.stderr[-2000:]}")
    return json.loads(r.stdout.strip().splitlines()[-1])


def host_cores() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def cpu_baseline(workload: str, nrhs: int, iterations: int, samples: int = 1) -> dict:
    """The oracle's solves/s on this host, shared by the GPU arm's cpu_baseline and --impl
    reference.  Run twice in fresh interpreters: numpy's BLAS on one thread (`samples` timed
    samples) and on every core (one sample).  On every core the many small dense operations of
    the lower levels run far slower than on one (thread start-up per call), so the reported
    value is the faster configuration's median, with the threads it used; both are listed."""
    cores = host_cores()
    one = _oracle_subprocess(workload, nrhs, iterations, 1, samples)
    allc = _oracle_subprocess(workload, nrhs, iterations, cores, 1) if cores > 1 else one
    v1 = statistics.median(r["solves_per_s"] for r in one["runs"])
    va = statistics.median(r["solves_per_s"] for r in allc["runs"])
    best, used, runs = (v1, 1, one["runs"]) if v1 >= va else (va, cores, allc["runs"])
    r0 = runs[len(runs) // 2]
    return {"value": best, "unit": "solves/s", "cores": used, "kind": "oracle",
            "sample": (f"per sample: {r0['leaf_sample']} leaf maps (16 of them a 4x4 block) scaled to all "
                       f"elements; every pair merge of levels 1-4 of that block on real maps, one pair merge per "
                       f"higher level on random children of the true sizes, each scaled by the pairs of its "
                       f"level (levels 9 and up: the merge timed once, in the warm-up sample); one FP64 matvec + one "
                       f"V-cycle's pair sweeps + the coarse GMRES steps for one RHS "
                       f"x {iterations} FGMRES iterations x {one['nrhs']} RHS; {len(runs)} sample(s) of about "
                       f"{r0['measured_s']:.1f} s of CPU work each, median; numpy/LAPACK"),
            "value_1_thread": v1, "value_all_cores": va, "host_cores": cores, "samples": [r["solves_per_s"] for r in runs],
            "phases_s": {"leaves": r0["t_leaf"], "merges": r0["t_merge"], "solve_per_rhs": r0["t_solve_per_rhs"]},
            "extrapolated": True}


# ---------------------------------------------------------------------------- batching / serving
def run_table1(args, prec):
    """Memory-time trade-off of section 5 (Table 1) on the 64x64, N = 16, kappa = 100 problem, one
    right-hand side as in the paper: for #levels = L_exact + 1 = 2..12 the device bytes of the tree
    beyond the leaf maps (PMem) and the merge time (Bt), and FGMRES iterations (It) and solve time
    (St) for gamma = 1 with 4, 5, 6 coarse GMRES steps and gamma = 2 with 2, 3, 4 (up to #levels 7,
    as in the paper), plus direct HPS (exact coarse level) and unpreconditioned GMRES.  Times are
    CUDA events on the library's stream; each solve runs once untimed first (V-cycle graph
    capture)."""
    import torch

    from paper_2511_00735_gb300 import hps as H
    from paper_2511_00735_gb300 import inputs

    nrhs = args.nrhs or 1
    prob = inputs.fp64_64x64(seed=1, nrhs=nrhs)
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

    def solve(ci, restart=60, max_outer=20):
        return s.gmres_solve(t_dev, tol=args.tol, inner_iters=ci, restart=restart, max_outer=max_outer, out=g_dev,
                             raise_on_notconv=False)[1]

    rows = []

    def emit(row):
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)

    # unpreconditioned FGMRES (PMem 0, Bt 0)
    solve(-1, 60, 40)
    st, info = ev_ms(lambda: solve(-1, 60, 40))
    emit({"levels": 0, "coarse": "none (unpreconditioned)", "gamma": 0, "pmem_bytes": 0, "bt_ms": 0.0,
          "it": info["outer_iterations"], "converged": info["converged"], "st_ms": st,
          "max_rel_residual": info["max_rel_residual"]})
    cases = [(lx, False) for lx in range(1, s.levels)] + [(s.levels - 1, True)]
    for lx, exact in cases:
        s.release_workspace()
        s.set_gamma(1)
        s.merge_levels(lx, exact_coarse=exact)  # plan for this depth, then the timed build
        bt, _ = ev_ms(lambda: s.merge_levels(lx, exact_coarse=exact))
        held = s.bytes_held()
        cols = [(1, 0)] if exact else [(1, ci) for ci in (4, 5, 6)] + (
            [(2, ci) for ci in (2, 3, 4)] if lx + 1 <= 7 else [])
        for gamma, ci in cols:
            s.set_gamma(gamma)
            solve(ci)  # first solve of a configuration captures the V-cycle graph
            st, info = ev_ms(lambda: solve(ci))
            emit({"levels": lx + 1, "L_exact": lx, "coarse": "exact" if exact else f"{ci} c.i.", "gamma": gamma,
                  "pmem_bytes": held - leaf_bytes, "bytes_held_tree": held, "bt_ms": bt,
                  "it": info["outer_iterations"], "converged": info["converged"], "st_ms": st,
                  "max_rel_residual": info["max_rel_residual"]})
    s.set_gamma(1)
    s.close()
    return {"metric": "memory-time trade-off (section 5, Table 1): PMem, Bt, It, St by levels, coarse steps, gamma",
            "value": None, "unit": None, "n_gpus": 1, "dtype": "f64+f32" if prec else "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS["scattering64"][0].replace(
                "16 plane-wave RHS, L_exact=10, 5 coarse GMRES steps",
                f"{nrhs} plane-wave RHS, L_exact, coarse steps and gamma swept"),
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


# ---------------------------------------------------------------------------- one phase (profilers)
def run_phase(args):
    """One phase of a workload in isolation, for ncu: `leaf` (R leaf builds), `merge` (leaves, then
    R merge-tree builds), `matvec` (R FP64 skeleton matvecs), `mixed_matvec` (R of the mixed
    path's Arnoldi matvecs, --mv tensor|simt), `precond` (R preconditioner
    applications), `solve` (one FGMRES solve on a built tree) or `step` (R whole bench steps
    after one untimed step).  --nx 32 runs the 32x32, N = 16, kappa = 50 problem."""
    import torch

    from paper_2511_00735_gb300 import hps as H
    from paper_2511_00735_gb300 import inputs

    prec = H.HPS_MIXED if args.precision == "mixed" else H.HPS_FP64
    if args.nx in (0, 128):
        prob = make_problem("scattering128", 2, args.nrhs)
    elif args.nx == 64:
        prob = make_problem("scattering64", 1, args.nrhs)
    else:
        L = 2 * int(round(np.log2(args.nx)))
        prob = inputs.single_bump(args.nx, 16, 100.0 * args.nx / 64.0, args.nrhs, seed=1, L_exact=max(L - 2, 0))
    s = H.Solver(0)
    s.set_autotune(H.TUNE_ON if args.autotune == "on" else H.TUNE_OFF)  # tuned in the untimed first call
    t = H.setup(s, prob, prec, build=False)
    td = torch.from_numpy(t).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info = None
    prof = torch.cuda.profiler  # the repeated phase is bracketed by cudaProfilerStart / Stop
    if args.phase == "leaf":
        s.build_leaves(prec)
        torch.cuda.synchronize()
        prof.start()
        for _ in range(args.repeat):
            s.build_leaves(prec)
    else:
        s.build_leaves(prec)
        if args.phase == "merge":
            s.merge_levels(prob.L_exact)
            torch.cuda.synchronize()
            prof.start()
            for _ in range(args.repeat):
                s.merge_levels(prob.L_exact)
        elif args.phase == "matvec":
            x = torch.randn((prob.nrhs, s.n_skel), dtype=torch.complex128, device="cuda")
            s.matvec(x)
            torch.cuda.synchronize()
            prof.start()
            for _ in range(args.repeat):
                s.matvec(x)
        elif args.phase == "mixed_matvec":
            # the mixed path's Arnoldi matvec (FP32 input, double-float product) by the chosen method
            s.set_arnoldi_matvec(H.MV_TENSOR if args.mv == "tensor" else H.MV_SIMT)
            x = torch.randn((prob.nrhs, s.n_skel), dtype=torch.complex128, device="cuda")
            s.matvec_mixed(x)
            torch.cuda.synchronize()
            prof.start()
            for _ in range(args.repeat):
                s.matvec_mixed(x)
        elif args.phase == "step":
            # one whole bench step (coefficient, leaves, merges, FGMRES) after one untimed step
            X, Y = s.node_coords()
            b = torch.from_numpy(np.ascontiguousarray(inputs.eval_b(prob.bumps, X, Y))).cuda()

            def one():
                s.set_coeff(prob.kappa, b, prob.eta)
                s.build_leaves(prec)
                s.merge_levels(prob.L_exact)
                return s.gmres_solve(td, tol=args.tol, inner_iters=prob.inner_iters, restart=args.restart,
                                     max_outer=args.max_outer, raise_on_notconv=False)[1]
            one()
            torch.cuda.synchronize()
            prof.start()
            for _ in range(args.repeat):
                info = one()
        elif args.phase == "precond":
            s.merge_levels(prob.L_exact)
            r = torch.randn((prob.nrhs, s.n_skel), dtype=torch.complex128, device="cuda")
            s.precond_apply(r, prob.inner_iters)
            torch.cuda.synchronize()
            prof.start()
            for _ in range(args.repeat):
                s.precond_apply(r, prob.inner_iters)
        else:
            s.merge_levels(prob.L_exact)
            torch.cuda.synchronize()
            prof.start()
            _, info = s.gmres_solve(td, tol=args.tol, inner_iters=prob.inner_iters)
    torch.cuda.synchronize()
    prof.stop()
    line = {"phase": args.phase, "workload": prob.name, "repeat": args.repeat,
            "wall_s": time.perf_counter() - t0, "bytes_held": s.bytes_held()}
    if info:
        line.update(iterations=info["outer_iterations"], max_rel_residual=info["max_rel_residual"])
    if args.autotune == "on":
        line["autotune"] = H.autotune_table().splitlines()
    s.close()
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- main
def pct(xs, p):
    xs = sorted(xs)
    if not xs:
        return None
    k = (len(xs) - 1) * p / 100.0
    lo, hi = int(np.floor(k)), int(np.ceil(k))
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--nrhs", type=int, default=0, help="right-hand sides (default: the workload's)")
    ap.add_argument("--outer", default="default", choices=["default", "fp64", "df64"],
                    help="outer FGMRES arithmetic (default: df64 for mixed, fp64 for fp64)")
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--restart", type=int, default=20, help="FGMRES restart length (the paper's Table 1: 60)")
    ap.add_argument("--max-outer", type=int, default=40, help="FGMRES restart cycles at most")
    ap.add_argument("--autotune", default="on", choices=["on", "off"],
                    help="tile autotuner of the tensor-core GEMMs (tuned in the warm-up steps)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison run")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-extra", action="store_true", help="skip the 64x64 extra line")
    ap.add_argument("--workload", default="scattering128",
                    choices=["scattering128", "scattering64", "batch", "serve", "table1", "phase"],
                    help="scattering128 (default) / scattering64: the timed step above; batch: the 512-problem "
                         "mix; serve: a Poisson stream; table1: the memory-time trade-off over exact levels and "
                         "coarse steps; phase: one phase in isolation (for profilers)")
    ap.add_argument("--phase", default="leaf",
                    choices=["leaf", "merge", "matvec", "mixed_matvec", "precond", "solve", "step"])
    ap.add_argument("--mv", default="tensor", choices=["tensor", "simt"], help="phase mixed_matvec: method")
    ap.add_argument("--nx", type=int, default=0, help="phase: element grid (0: 128)")
    ap.add_argument("--repeat", type=int, default=1, help="phase: repetitions")
    ap.add_argument("--count", type=int, default=0, help="problems (batch) or requests (serve)")
    ap.add_argument("--rate", type=float, default=200.0, help="serve: arrivals per second")
    ap.add_argument("--slots", type=int, default=8, help="batch slots / serve workers")
    ap.add_argument("--serve-timeout", type=float, default=240.0, help="serve: stop waiting after this many seconds")
    ap.add_argument("--oracle-sample", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--oracle-iterations", type=int, default=0, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_sample:  # internal: the CPU oracle's bounded samples in a pinned-thread subprocess
        wl = args.oracle_sample
        r = oracle_samples(wl, args.nrhs or WORKLOADS[wl][1], args.oracle_iterations or ORACLE_ITERATIONS[wl],
                           args.steps)
        print(json.dumps(r), flush=True)
        return
    if args.workload == "phase":
        if not args.nrhs:
            args.nrhs = 32 if args.nx in (0, 128) else 16
        return run_phase(args)
    if args.workload not in WORKLOADS:
        return run_systems(args)
    desc, default_nrhs, base_seed = WORKLOADS[args.workload]
    if not args.nrhs:
        args.nrhs = default_nrhs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        iters = ORACLE_ITERATIONS[args.workload]
        base = cpu_baseline(args.workload, args.nrhs, iters, samples=args.steps)
        v = base["value"]
        ms_step = 1e3 * args.nrhs / v
        line = {"metric": METRIC, "value": v, "unit": "solves/s",
                "impl": "reference", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": desc, "global_batch": args.nrhs, "parallelism": "replicas",
                           "l2": "host run (no GPU)"},
                "latency_ms": {"p50": ms_step, "p99": ms_step,
                               "note": "every solve of a step arrives at its start and completes at its end; "
                                       "extrapolated step time of the sampled oracle"},
                "extrapolated": True,
                "cpu_baseline": base,
                "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    dist = None
    if world > 1:
        import torch.distributed as tdist

        tdist.init_process_group("nccl")
        dist = tdist
    r = run_gpu(args, rank, world, local_rank, dist)
    extra = None
    if world == 1 and args.workload == "scattering128" and not args.no_extra:
        ex_args = argparse.Namespace(**vars(args))
        ex_args.workload, ex_args.nrhs, ex_args.no_fp64 = "scattering64", 16, True
        ex_args.steps, ex_args.warmup = max(3, min(args.steps, 10)), 3
        rx = run_gpu(ex_args, rank, world, local_rank, dist)
        extra = {"workload": WORKLOADS["scattering64"][0], "value": rx["value"], "unit": "solves/s",
                 "steps": ex_args.steps, "ms_per_step": rx["ms"] / ex_args.steps, "iterations": rx["its"],
                 "max_rel_residual": rx["res"], "converged_per_step": rx["conv"],
                 "e2e_value": rx["e2e_conv"] / (rx["e2e_ms"] / 1e3),
                 "warm_value": rx["warm_conv"] / (rx["warm_ms"] / 1e3)}
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    prob = r["prob"]
    peaks = load_peaks()
    nrhs = prob.nrhs
    prof = r["prof"]
    E, N = prob.nx * prob.nx, prob.N
    # the dominant kernel of a step: the bf16x3 sweep GEMM (2 L_exact launches per V-cycle, about a
    # fifth of the step), timed launch by launch in the pass after the timed region; the leaf
    # kernel (one launch per step) and the V-cycle as a whole are reported beside it
    kern = r.get("kern")
    roof = None
    if kern and kern["sweep"][1]:
        ms_k, n_k, by_k, fl_k = kern["sweep"]
        hbm = peaks.get("hbm_gbs", 6800.0)
        per = ms_k / n_k
        bpl = by_k / n_k
        calls = kern["precond_calls_per_step"]
        roof = {"kernel": "tcb_gemm_kernel (bf16x3 sweep products of the V-cycle, every merge level, up and down)",
                "bound": "hbm", "achieved": bpl / (per / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": bpl / (per / 1e3) / 1e9 / hbm,
                "traffic": SWEEP_TRAFFIC_RATIO * bpl if SWEEP_TRAFFIC_RATIO else None,
                "traffic_unit": "bytes per launch (ncu dram read + write / algorithmic bytes of a 64x64 capture x "
                                "this launch's algorithmic bytes)",
                "algorithmic_bytes_per_launch": bpl, "ms_per_launch": per, "launches_timed": n_k,
                "bytes_model": "per product: the tiled operator (8 B per complex entry), B, C0 when present and C, "
                               "each once",
                "timing": f"CUDA events around each launch on the launching stream, {kern['applies']} direct "
                          "V-cycle applications of the bench tree after the timed region",
                "share_of_step_est": ms_k / kern["applies"] * calls * args.steps / r["ms"],
                "peak_source": "measured" if not peaks.get("fallback") else "fallback 6.8 TB/s"}
    mg = None
    if kern and kern["merge_gemm"][1]:
        ms_m, n_m, by_m, fl_m = kern["merge_gemm"]
        tf32 = peaks.get("bf16_tflops", 1900.0) * TF32_OVER_BF16
        mg = {"kernel": "merge GEMMs (3xTF32 tc_gemm_kernel above 64 rows, SIMT below)", "bound": "tensor",
              "achieved": fl_m / (ms_m / 1e3) / 1e12, "peak": tf32, "unit": "TFLOP/s",
              "frac": fl_m / (ms_m / 1e3) / 1e12 / tf32, "launches": n_m, "ms_per_merge_phase": ms_m,
              "flops_model": "8 m n k per complex product (3xTF32 issues three tf32 MMAs per product)",
              "peak_source": "measured bf16 x nominal tf32/bf16 ratio (1.1/2.25)"}
    leaf_ms, leaf_launch, leaf_calls = prof["leaf"]
    leaf_roof = None
    if leaf_calls:
        per = leaf_ms / leaf_calls
        lit = leaf_flops_paper(N) * E
        ex = leaf_flops(N) * E
        leaf_roof = {"kernel": "leaf_ir_kernel (leaf ItI maps: FP32 factor, double-float refinement and inverse)",
                "bound": "alu", "achieved": lit / (per / 1e3) / 1e12, "peak": FP32_PEAK_NOMINAL / 1e12,
                "unit": "TFLOP/s", "frac": lit / (per / 1e3) / FP32_PEAK_NOMINAL,
                "traffic": LEAF_TRAFFIC_BYTES_PER_ELEMENT * E if LEAF_TRAFFIC_BYTES_PER_ELEMENT else None,
                "traffic_unit": "bytes per launch (ncu dram read + write per element x elements)",
                "algorithmic_flops_per_launch": lit, "ms_per_launch": per,
                "flops_model": "paper-literal dense complex LU of the (N+1)^2-4 node element matrix with 4q "
                               "right-hand sides, 8 (n_L^3/3 + n_L^2 n_G) per element",
                "executed_fp32_pipe_flops_per_launch": ex,
                "executed_rate_tflops": ex / (per / 1e3) / 1e12,
                "peak_source": "FP32 pipes from unit counts and clock: 152 SMs x 128 lanes x 2 (FMA) x "
                               "2.07 GHz = 80.5 TFLOP/s (no FP32 entry in the measured peaks)",
                "share_of_step": leaf_ms / r["ms"]}
    pre_ms, _, pre_calls = prof["precond"]
    vc = None
    if pre_calls:
        vb = vcycle_bytes(prob.nx, N, prob.L_exact, nrhs, prob.inner_iters)
        per = pre_ms / pre_calls
        hbm = peaks.get("hbm_gbs", 6800.0)
        vc = {"kernel": "V-cycle (one CUDA graph: sweep GEMMs, coarse GMRES, gathers)", "bound": "hbm",
              "achieved": vb["bytes"] / (per / 1e3) / 1e9, "peak": hbm, "unit": "GB/s",
              "frac": vb["bytes"] / (per / 1e3) / 1e9 / hbm, "traffic": None,
              "algorithmic_bytes_per_launch": vb["bytes"], "operator_bytes": vb["operator_bytes"],
              "vector_bytes": vb["vector_bytes"], "ms_per_launch": per, "launches_per_step": pre_calls / args.steps,
              "share_of_step": pre_ms / r["ms"],
              "peak_source": "measured" if not peaks.get("fallback") else "fallback 6.8 TB/s"}
    cpu = None
    if not args.no_cpu and world == 1:
        cpu = cpu_baseline(args.workload, nrhs, r["its"], samples=1)
    laps = r["laps"]
    line = {
        "metric": METRIC,
        "value": r["value"], "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": r["ms"] / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64+f32" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": desc, "global_batch": nrhs * world, "precision": args.precision,
                   "autotune": args.autotune,
                   "outer": r["outer"], "tol": args.tol, "restart": args.restart,
                   "parallelism": "replicas" if world > 1 else "single",
                   "residual": "FP64 (FP64 leaf maps and norms) at every restart and for the returned solution",
                   "l2": "inputs larger than L2: leaf maps 0.94 GB, merge tree ~6 GB, Krylov basis ~30 GB per step"
                   if args.workload == "scattering128" else
                   "inputs larger than L2: leaf maps 236 MB, merge tree ~1.3 GB, Krylov basis 3.8 GB per step"},
        "latency_ms": {"p50": pct(laps, 50), "p99": pct(laps, 99),
                       "note": "per-step device time: every solve of a step arrives at its start and completes at "
                               "its end (Poisson-arrival latencies: --workload serve)"},
        "iterations": r["its"], "max_rel_residual": r["res"], "converged": r["conv"],
        "e2e": {"value": r["e2e_conv"] / (r["e2e_ms"] / 1e3), "unit": "solves/s",
                "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"],
                "host_buffers": "page-locked numpy arrays (b and t in, g out) through hps_set_coeff / hps_gmres_solve",
                "wall_value": r["e2e_conv"] / (r["e2e_wall"] / 1e3)},
        "warm": {"value": r["warm_conv"] / (r["warm_ms"] / 1e3), "unit": "solves/s",
                 "latency_ms": {"p50": pct(r["warm_laps"], 50), "p99": pct(r["warm_laps"], 99)},
                 "note": "cached leaf maps and merge tree, solve phase only"},
        "warm_restart60": r["r60"],
        "fp64": r["fp64"],
        "gpu_launches": r["launches"],
        "phases_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "launches_per_step": {k: v[1] / args.steps for k, v in prof.items()},
        "roofline": roof,
        "roofline_vcycle": vc,
        "roofline_leaf": leaf_roof,
        "roofline_merge_gemm": mg,
        "autotune": {"mode": args.autotune, "table": r.get("tune_table", "").splitlines()},
        "cpu_baseline": cpu,
        "clocks": r["clk"],
        "peaks": {"hbm_gbs": peaks.get("hbm_gbs"), "bf16_tflops": peaks.get("bf16_tflops"),
                  "fp64_tflops_nominal": FP64_PEAK_NOMINAL / 1e12, "fallback": bool(peaks.get("fallback"))},
    }
    if extra:
        line["extra_64x64"] = extra
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
