"""Independent replicas across GPUs: seeding, the bracketed timed region, whole-job throughput.

The solve shards by independent problems (one process per GPU, each rank its own seeded
scattering problem), so the data path has no collective.  The only collectives are the
barrier on each side of a timed region and the max-reduction of the per-rank times; the
job's throughput is the units all ranks processed divided by the slowest rank's time.

`dist` is `torch.distributed` (or None for one process); `device` is where the reduction
tensor lives (the rank's CUDA device under NCCL, "cpu" under gloo); `sync` is called after
each barrier (the CUDA path passes `torch.cuda.synchronize`).
"""
from __future__ import annotations

import time


def seed_for_rank(rank: int, base: int = 1) -> int:
    """Seed of rank `rank`'s problem: every replica solves a different seeded problem."""
    return base + rank


def barrier(dist=None, sync=None) -> None:
    if dist is not None:
        dist.barrier()
    if sync is not None:
        sync()


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    if dist is None:
        return float(x)
    import torch

    v = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(v, op=dist.ReduceOp.MAX)
    return float(v.item())


def sum_over_ranks(x: float, dist=None, device="cpu") -> float:
    if dist is None:
        return float(x)
    import torch

    v = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(v, op=dist.ReduceOp.SUM)
    return float(v.item())


class WallClock:
    """Host timer with the interface of `CudaEventClock` (for CPU ranks and tests)."""

    def start(self):
        self.t0 = time.perf_counter()
        self.marks = [self.t0]

    def lap(self):
        self.marks.append(time.perf_counter())

    def stop(self):
        self.t1 = time.perf_counter()

    def elapsed_ms(self) -> float:
        return (self.t1 - self.t0) * 1e3

    def laps_ms(self) -> list:
        return [(b - a) * 1e3 for a, b in zip(self.marks, self.marks[1:])]


class CudaEventClock:
    """CUDA events recorded on the stream the work is launched on (one more after each step,
    so the per-step device times are known too)."""

    def __init__(self, stream):
        import torch

        self.torch = torch
        self.stream = stream
        self.e0 = torch.cuda.Event(enable_timing=True)
        self.e1 = torch.cuda.Event(enable_timing=True)
        self.marks = []

    def start(self):
        self.e0.record(self.stream)
        self.marks = [self.e0]

    def lap(self):
        e = self.torch.cuda.Event(enable_timing=True)
        e.record(self.stream)
        self.marks.append(e)

    def stop(self):
        self.e1.record(self.stream)

    def elapsed_ms(self) -> float:  # valid once the stream has passed e1 (the closing barrier syncs)
        return self.e0.elapsed_time(self.e1)

    def laps_ms(self) -> list:
        return [a.elapsed_time(b) for a, b in zip(self.marks, self.marks[1:])]


def timed(fn, k: int, clock, dist=None, sync=None, device="cpu"):
    """Run `fn` k times between two barriers.

    Returns (max over ranks of the clock's milliseconds, max over ranks of the host wall
    milliseconds, the k outputs of this rank)."""
    barrier(dist, sync)
    w0 = time.perf_counter()
    clock.start()
    out = []
    for _ in range(k):
        out.append(fn())
        clock.lap()
    clock.stop()
    barrier(dist, sync)
    wall_ms = (time.perf_counter() - w0) * 1e3
    return max_over_ranks(clock.elapsed_ms(), dist, device), max_over_ranks(wall_ms, dist, device), out


def job_throughput(units_per_step: float, steps: int, world: int, ms: float) -> float:
    """Units per second of the whole job: every rank processes `units_per_step` per step."""
    return steps * units_per_step * world / (ms / 1e3)
