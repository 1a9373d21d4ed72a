"""Continuous-batching solve server on one GPU.

A request asks for the skeleton solution of one scattering problem for a few
plane-wave right-hand sides.  Problems are identified by a tree key (element
grid, GLL order, wavenumber, coefficient); the factorised merge tree of a key
is built once and kept on the device in its own libhps context (own CUDA
stream) while it is in use or until memory is needed (LRU among idle trees).

Workers (threads) repeatedly take the oldest waiting request and, with it,
every other waiting request for the same tree, up to `max_rhs` right-hand sides:
requests that arrived while that tree was busy join its next solve (continuous
batching), and different trees' solves overlap on the device on their own
streams.  A tree is admitted only when the device memory held by all live
contexts plus an estimate for the new one stays under `hbm_cap`.

Latency = completion time - arrival time (real clock).  run_stream() replays a
Poisson arrival stream and reports p50/p99 latency and solves/s.
"""
from __future__ import annotations

import collections
import math
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import hps as H
from . import inputs


@dataclass
class Request:
    rid: int
    prob: inputs.Problem          # its thetas are this request's right-hand sides
    arrival: float = 0.0          # seconds since the stream started
    done: float = -1.0
    g: np.ndarray | None = None
    info: dict = field(default_factory=dict)

    @property
    def key(self):
        p = self.prob
        return (p.nx, p.N, p.kappa, tuple((b.amp, b.cx, b.cy, b.gamma) for b in p.bumps), p.L_exact,
                p.inner_iters)


def tree_bytes_estimate(nx: int, N: int, nrhs: int, precision: int, restart: int = 60) -> int:
    """Device bytes of one context: leaf maps, merge tree and sweep operators, FGMRES workspace."""
    return tree_only_bytes(nx, N, precision) + krylov_bytes(nx, N, nrhs, restart)


def tree_only_bytes(nx: int, N: int, precision: int) -> int:
    """Leaf maps (FP64), stage maps, interface inverses and sweep operators (upper estimate)."""
    q = N - 1
    E = nx * nx
    leaf = E * (4 * q) ** 2 * 16
    cs = 16 if precision == H.HPS_FP64 else 8
    L = 2 * int(round(math.log2(nx)))
    return leaf + int(3.0 * L * E * (4 * q) ** 2 * cs) + (64 << 20)


def krylov_bytes(nx: int, N: int, nrhs: int, restart: int = 60) -> int:
    """Per-solve workspace: FGMRES basis V and Z, sweep vectors of every stage, staging, and the
    double-float copy of the leaf maps that the mixed path's outer iteration reads (an upper
    bound for both outer arithmetics)."""
    rows = nx * nx * 4 * (N - 1)
    return (2 * restart + 8) * rows * nrhs * 16 + 4 * rows * nrhs * 16 + rows * 4 * (N - 1) * 16 + (32 << 20)


class _Tree:
    def __init__(self, key, solver: H.Solver, stream):
        self.key = key
        self.solver = solver
        self.stream = stream
        self.busy = False
        self.last_used = time.perf_counter()
        self.ready = False
        self.tree_bytes = 0


class Server:
    def __init__(self, device: int = 0, workers: int = 4, precision: int = H.HPS_MIXED, tol: float = 1e-10,
                 hbm_cap: float = 150e9, max_rhs: int = 64, restart: int = 60, max_outer: int = 20,
                 torch_module=None):
        # torch_module: the device runtime (torch by default; the host-logic tests pass a stand-in
        # with the few torch.cuda calls used here)
        if torch_module is None:
            import torch as torch_module
        torch = torch_module
        self.torch = torch
        self.device = device
        self.precision = precision
        self.tol, self.restart, self.max_outer = tol, restart, max_outer
        self.hbm_cap = hbm_cap
        self.max_rhs = max_rhs
        self.lock = threading.Condition()
        self.pending = collections.deque()
        self.trees = {}
        self.stop = False
        self.completed = []
        self.peak_bytes = 0
        self.evictions = 0
        self.inflight = 0  # bytes reserved by running jobs
        torch.cuda.empty_cache()
        self.base = torch.cuda.memory_reserved(device)  # held by the process before the server started
        self.workers = [threading.Thread(target=self._worker, daemon=True) for _ in range(workers)]
        for w in self.workers:
            w.start()

    # ---- public ------------------------------------------------------------
    def submit(self, req: Request):
        with self.lock:
            self.pending.append(req)
            self.lock.notify_all()

    def drain(self, n_expected: int, timeout: float = 3600.0, progress=None):
        t0 = time.perf_counter()
        last = t0
        with self.lock:
            while len(self.completed) < n_expected and time.perf_counter() - t0 < timeout:
                self.lock.wait(0.05)
                if progress and time.perf_counter() - last > 10.0:
                    last = time.perf_counter()
                    progress(f"[serve] t={last - t0:.0f}s done={len(self.completed)}/{n_expected} "
                             f"pending={len(self.pending)} trees={len(self.trees)} "
                             f"busy={sum(t.busy for t in self.trees.values())} held={self._held() / 1e9:.1f}GB")
        return list(self.completed)

    def close(self):
        with self.lock:
            self.stop = True
            self.lock.notify_all()
        for w in self.workers:
            w.join()
        for t in self.trees.values():
            t.solver.close()
        self.trees.clear()

    # ---- internals ---------------------------------------------------------
    def _held(self) -> int:
        """Device bytes in use: built trees (measured after their build) plus what running jobs reserved;
        never less than what torch's allocator holds."""
        model = sum(t.tree_bytes for t in self.trees.values() if t.ready) + self.inflight
        return max(model, self.torch.cuda.memory_reserved(self.device) - self.base)

    def _pick(self):
        """Under the lock: choose the next job (tree, requests) or None."""
        if not self.pending:
            return None
        # oldest request whose tree is not busy
        for idx, r in enumerate(self.pending):
            t = self.trees.get(r.key)
            if t is not None and t.busy:
                continue
            batch, nrhs = [], 0
            # right-hand sides per solve call: at most max_rhs and a Krylov workspace of about 16 GB;
            # a batch larger than that (one big request) is solved in consecutive chunks
            per_rhs = krylov_bytes(r.prob.nx, r.prob.N, 1, self.restart)
            chunk = max(1, min(self.max_rhs, int(16e9 // per_rhs)))
            cap_rhs = max(r.prob.nrhs, chunk)
            for r2 in list(self.pending):
                if r2.key == r.key and nrhs + r2.prob.nrhs <= cap_rhs:
                    batch.append(r2)
                    nrhs += r2.prob.nrhs
            need = krylov_bytes(r.prob.nx, r.prob.N, min(nrhs, chunk), self.restart)
            if t is None:
                need += tree_only_bytes(r.prob.nx, r.prob.N, self.precision)
            while self._held() + need > self.hbm_cap:
                idle = [x for x in self.trees.values() if not x.busy and x.ready and x is not t]
                if idle:
                    victim = min(idle, key=lambda x: x.last_used)
                    victim.solver.close()
                    del self.trees[victim.key]
                    self.evictions += 1
                    continue
                model = sum(x.tree_bytes for x in self.trees.values() if x.ready) + self.inflight
                if self.torch.cuda.memory_reserved(self.device) - self.base > model + need:
                    self.torch.cuda.empty_cache()  # return cached blocks, then re-check
                    if self._held() + need <= self.hbm_cap:
                        break
                return None  # wait for running jobs to release memory
            if t is None:
                stream = self.torch.cuda.Stream(self.device)
                t = _Tree(r.key, H.Solver(self.device, stream=stream), stream)
                self.trees[r.key] = t
            t.job_bytes = need
            t.chunk = chunk
            self.inflight += need
            t.busy = True
            for r2 in batch:
                self.pending.remove(r2)
            return t, batch
        return None

    def _fail_oldest(self, e):
        """Under the lock: report the oldest pending request as failed with the error e."""
        if not self.pending:
            return
        r = self.pending.pop(0)
        r.info = {"error": repr(e), "rel_residual": [float("inf")], "batched_with": 1}
        r.done = time.perf_counter() - self.t_origin
        self.completed.append(r)
        self.lock.notify_all()

    def _worker(self):
        while True:
            with self.lock:
                job = None
                while job is None:
                    if self.stop:
                        return
                    try:
                        job = self._pick()
                    except Exception as e:  # a context that cannot be created fails its requests
                        self._fail_oldest(e)
                        job = None
                    if job is None:
                        self.lock.wait(0.01)
            tree, batch = job
            try:
                self._run(tree, batch)
            except Exception as e:  # report on the requests instead of losing them
                now = time.perf_counter() - self.t_origin
                with self.lock:
                    for r in batch:
                        r.info = {"error": repr(e), "rel_residual": [float("inf")], "batched_with": len(batch)}
                        r.done = now
                        self.completed.append(r)
            finally:
                with self.lock:
                    self.inflight -= tree.job_bytes
                    tree.job_bytes = 0
                    tree.busy = False
                    # the caching allocator keeps freed blocks per stream; hand them back when over the cap
                    if self.torch.cuda.memory_reserved(self.device) - self.base > self.hbm_cap:
                        self.torch.cuda.empty_cache()
                    tree.last_used = time.perf_counter()
                    self.peak_bytes = max(self.peak_bytes, self._held())
                    self.lock.notify_all()

    def _run(self, tree: _Tree, batch):
        s = tree.solver
        prob = batch[0].prob
        with self.torch.cuda.stream(tree.stream):
            if not tree.ready:
                s.mesh(prob.nx, prob.N)
                X, Y = s.node_coords()
                s.set_coeff(prob.kappa, inputs.eval_b(prob.bumps, X, Y), prob.eta)
                s.build_leaves(self.precision)
                s.merge_levels(prob.L_exact)
                bx, by, bnx, bny = s.boundary_points()
                tree.bdry = (bx, by, bnx, bny)
                tree.tree_bytes = s.bytes_held()
                tree.ready = True
            bx, by, bnx, bny = tree.bdry
            thetas = [th for r in batch for th in r.prob.thetas]
            t = np.ascontiguousarray(np.stack([inputs.plane_wave_impedance(th, prob.kappa, prob.eta, bx, by, bnx, bny)
                                               for th in thetas]))
            gs, its, res = [], [], []
            for c0 in range(0, len(thetas), tree.chunk):
                g, info = s.gmres_solve(np.ascontiguousarray(t[c0:c0 + tree.chunk]), tol=self.tol,
                                        inner_iters=prob.inner_iters, restart=self.restart, max_outer=self.max_outer,
                                        raise_on_notconv=False)
                gs.append(g)
                its += info["iterations"]
                res += info["rel_residual"]
            s.release_workspace()
            g = np.concatenate(gs)
            info = {"iterations": its, "rel_residual": res}
        now = time.perf_counter() - self.t_origin
        k = 0
        with self.lock:
            for r in batch:
                n = r.prob.nrhs
                r.g = g[k:k + n]
                r.info = {"rel_residual": info["rel_residual"][k:k + n], "iterations": info["iterations"][k:k + n],
                          "batched_with": len(batch)}
                r.done = now
                k += n
                self.completed.append(r)


def poisson_stream(count: int, rate: float, seed: int = 5, big_fraction: float = 0.1, rhs_range=(1, 64),
                   mix_trees: int = 32, big_trees: int = 2):
    """Requests: `count` Poisson arrivals at `rate`/s; each picks one of `mix_trees` problems of the
    batching mix (or, with probability big_fraction, one of `big_trees` 128x128 N=16 kappa=200 jobs)
    and asks for U{rhs_range} plane waves of it."""
    rng = inputs.SplitMix64(seed)
    mix = inputs.batch_mix(mix_trees, seed + 1)
    big = [inputs.multi_bump(128, 16, 200.0, 8, 1, seed + 100 + i, L_exact=12) for i in range(big_trees)]
    reqs, t = [], 0.0
    for i in range(count):
        t += -math.log(1.0 - rng.uniform()) / rate
        base = big[rng.randint(0, big_trees - 1)] if rng.uniform() < big_fraction else mix[rng.randint(0, mix_trees - 1)]
        nrhs = rng.randint(*rhs_range)
        thetas = [rng.uniform(0.0, 2.0 * math.pi) for _ in range(nrhs)]
        p = inputs.Problem(nx=base.nx, N=base.N, kappa=base.kappa, eta=base.eta, bumps=base.bumps, thetas=thetas,
                           L_exact=base.L_exact, inner_iters=base.inner_iters, name=base.name)
        reqs.append(Request(i, p, t))
    return reqs


def run_stream(reqs, server: Server, time_scale: float = 1.0, timeout: float = 3600.0, progress=None):
    """Replay the arrivals (arrival times multiplied by time_scale) and wait for every result."""
    t0 = time.perf_counter()
    server.t_origin = t0
    for r in reqs:
        r.arrival = r.arrival * time_scale
        delay = r.arrival - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        server.submit(r)
    done = server.drain(len(reqs), timeout, progress)
    makespan = time.perf_counter() - t0
    lat = np.array([r.done - r.arrival for r in done])
    ok = [r for r in done if max(r.info["rel_residual"]) <= server.tol]
    solves = sum(r.prob.nrhs for r in ok)
    res = max((max(r.info["rel_residual"]) for r in ok), default=0.0)
    return {"requests": len(done), "requests_submitted": len(reqs), "requests_converged": len(ok), "solves": solves,
            "seconds": makespan, "solves_per_s": solves / makespan,
            "p50_latency_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_latency_s": float(np.percentile(lat, 99)) if len(lat) else None,
            "max_rel_residual": res, "peak_device_bytes": server.peak_bytes,
            "mean_batch": float(np.mean([r.info["batched_with"] for r in done])) if done else None,
            "errors": sorted({r.info["error"][:300] for r in done if "error" in r.info})[:5]}
