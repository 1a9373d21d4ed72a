"""Batched solves of many independent scattering problems on one GPU.

Problems (paper_2511_00735_gb300.inputs.Problem) of mixed element grids, GLL
orders, wavenumbers and right-hand-side counts run in waves of `slots`
problems.  Each slot is one libhps context with its own CUDA stream, reused
across problems (its mesh is rebuilt only when the shape changes).  Per wave:
the leaf ItI maps of every problem are built by hps_build_leaves_batch (one
kernel launch per GLL order over all elements of the wave), then each
problem's merges and FGMRES run on its slot's stream from a worker thread, so
the problems of a wave overlap on the device.  Results go to host numpy.
"""
from __future__ import annotations

import threading
import time

import numpy as np

from . import hps as H
from . import inputs


class BatchRunner:
    def __init__(self, device: int = 0, slots: int = 8, precision: int = H.HPS_MIXED, tol: float = 1e-10,
                 restart: int = 60, max_outer: int = 20, torch_module=None):
        # torch_module: the device runtime (torch by default; the host-logic tests pass a stand-in)
        if torch_module is None:
            import torch as torch_module
        torch = torch_module
        self.torch = torch
        self.device = device
        self.precision = precision
        self.tol, self.restart, self.max_outer = tol, restart, max_outer
        self.streams = [torch.cuda.Stream(device) for _ in range(slots)]
        self.solvers = [H.Solver(device, stream=st) for st in self.streams]
        self.shapes = [None] * slots

    def close(self):
        for s in self.solvers:
            s.close()

    def _prepare(self, i: int, prob: inputs.Problem):
        s = self.solvers[i]
        if self.shapes[i] != (prob.nx, prob.N):
            s.mesh(prob.nx, prob.N)
            self.shapes[i] = (prob.nx, prob.N)
        X, Y = s.node_coords()
        s.set_coeff(prob.kappa, inputs.eval_b(prob.bumps, X, Y), prob.eta)
        bx, by, bnx, bny = s.boundary_points()
        return np.ascontiguousarray(np.stack([inputs.plane_wave_impedance(th, prob.kappa, prob.eta, bx, by, bnx, bny)
                                              for th in prob.thetas]))

    def run(self, problems):
        """Solve every problem; returns a list of (g [nrhs][n_skel] complex128, info dict) in order."""
        out = [None] * len(problems)
        nslot = len(self.solvers)
        for w0 in range(0, len(problems), nslot):
            wave = list(range(w0, min(w0 + nslot, len(problems))))
            ts = [self._prepare(i, problems[j]) for i, j in enumerate(wave)]
            H.build_leaves_batch(self.solvers[:len(wave)], self.precision)
            errs = []

            def work(i, j):
                try:
                    s = self.solvers[i]
                    with self.torch.cuda.stream(self.streams[i]):
                        s.merge_levels(problems[j].L_exact)
                        g, info = s.gmres_solve(ts[i], tol=self.tol, inner_iters=problems[j].inner_iters,
                                                restart=self.restart, max_outer=self.max_outer,
                                                raise_on_notconv=False)
                    out[j] = (g, info)
                except Exception as e:  # reported after the wave
                    errs.append((j, e))

            threads = [threading.Thread(target=work, args=(i, j)) for i, j in enumerate(wave)]
            for th in threads:
                th.start()
            for th in threads:
                th.join()
            if errs:
                raise errs[0][1]
        return out


def solve_alone(prob: inputs.Problem, precision: int = H.HPS_MIXED, tol: float = 1e-10, device: int = 0):
    """One problem through a fresh context (reference for the batched results)."""
    s = H.Solver(device)
    t = H.setup(s, prob, precision)
    s.merge_levels(prob.L_exact)
    g, info = s.gmres_solve(t, tol=tol, inner_iters=prob.inner_iters, raise_on_notconv=False)
    s.close()
    return g, info


def run_mix(count: int = 512, seed: int = 3, slots: int = 8, precision: int = H.HPS_MIXED, device: int = 0):
    """The batching workload: `count` problems from inputs.batch_mix; returns timing and accuracy."""
    import torch

    probs = inputs.batch_mix(count, seed)
    br = BatchRunner(device, slots, precision)
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    res = br.run(probs)
    torch.cuda.synchronize(device)
    dt = time.perf_counter() - t0
    br.close()
    nsolves = sum(p.nrhs for p in probs)
    conv = sum(info["converged"] for _, info in res)
    conv_res = [r for _, info in res for r in info["rel_residual"] if r <= 1e-10]
    stalled = [(p.nx, p.N, round(p.kappa, 1)) for p, (_, info) in zip(probs, res) if info["converged"] < p.nrhs]
    return {"problems": count, "solves": nsolves, "converged_solves": conv, "seconds": dt,
            "solves_per_s": conv / dt, "max_rel_residual_converged": max(conv_res) if conv_res else None,
            "not_converged_problems": stalled,
            "max_iterations": max(info["outer_iterations"] for _, info in res)}
