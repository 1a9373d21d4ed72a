"""Seeded synthetic workloads for the Helmholtz scattering problems.

This module draws the random numbers of a workload (bump parameters, plane-wave
angles) and evaluates the *problem data* of the model problem (the coefficient
b(x) and the incident plane wave and its impedance trace) at points the caller
supplies.  It holds none of the solver's arithmetic: no GLL rule, no element
operator, no skeleton index map.  Both the CPU oracle and the CUDA path take
their inputs from here.

Model problem (paper section 2, eq. diffhelm):
    -Lap u - kappa^2 (1 - b(x)) u = s   in (0,1)^2,
    du/dn + i eta u = t                  on the boundary, eta = kappa.

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), mapped to doubles in [0, 1)
with the top 53 bits.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 counter-based generator (64-bit state, golden-gamma step)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        u = (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def choice(self, items):
        return items[self.next_u64() % len(items)]

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive)."""
        return lo + int(self.next_u64() % (hi - lo + 1))


@dataclass
class Bump:
    """One Gaussian bump a * exp(-gamma * |x - c|^2)."""

    amp: float
    cx: float
    cy: float
    gamma: float


@dataclass
class Problem:
    """One scattering problem: mesh, order, wavenumber, coefficient, RHS angles."""

    nx: int
    N: int
    kappa: float
    eta: float
    bumps: list
    thetas: list
    L_exact: int = 0
    inner_iters: int = 5
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def ny(self) -> int:
        return self.nx

    @property
    def nrhs(self) -> int:
        return len(self.thetas)


def eval_b(bumps, x, y):
    """Coefficient b(x, y) = sum of Gaussian bumps, evaluated at arrays x, y."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    out = np.zeros(np.broadcast(x, y).shape)
    for bp in bumps:
        out += bp.amp * np.exp(-bp.gamma * ((x - bp.cx) ** 2 + (y - bp.cy) ** 2))
    return out


def plane_wave(theta, kappa, x, y):
    """Incident plane wave exp(i kappa d.x), d = (cos theta, sin theta)."""
    d0, d1 = math.cos(theta), math.sin(theta)
    return np.exp(1j * kappa * (d0 * np.asarray(x) + d1 * np.asarray(y)))


def plane_wave_impedance(theta, kappa, eta, x, y, n0, n1):
    """Impedance trace du/dn + i eta u of the plane wave at points with outward normal (n0, n1)."""
    d0, d1 = math.cos(theta), math.sin(theta)
    u = plane_wave(theta, kappa, x, y)
    return 1j * (kappa * (d0 * np.asarray(n0) + d1 * np.asarray(n1)) + eta) * u


# ---------------------------------------------------------------------------
# Workloads.  Sizes follow the paper's Gaussian-bump scattering experiment
# (section 5): degree-16 elements on a square grid, one or several bumps,
# plane-wave impedance data.
# ---------------------------------------------------------------------------
PAPER_BUMP = Bump(1.5, 0.5, 0.5, 160.0)


def _levels(nx: int) -> int:
    k = int(round(math.log2(nx)))
    assert (1 << k) == nx, "element grid must be 2^k x 2^k"
    return 2 * k


def small_4x4(seed: int = 0) -> Problem:
    """4x4 elements, N=8, kappa=eta=10, the paper's bump, one plane wave."""
    rng = SplitMix64(seed)
    theta = rng.uniform(0.0, 2.0 * math.pi)
    return Problem(nx=4, N=8, kappa=10.0, eta=10.0, bumps=[PAPER_BUMP],
                   thetas=[theta], L_exact=2, inner_iters=5, name="4x4_N8_k10")


def single_bump(nx: int, N: int, kappa: float, nrhs: int, seed: int,
                L_exact: int | None = None, inner_iters: int = 5, name: str = "") -> Problem:
    """One bump, centre U[0.3,0.7]^2, amplitude U[0.5,1.5], the paper's width 160."""
    rng = SplitMix64(seed)
    cx = rng.uniform(0.3, 0.7)
    cy = rng.uniform(0.3, 0.7)
    amp = rng.uniform(0.5, 1.5)
    thetas = [rng.uniform(0.0, 2.0 * math.pi) for _ in range(nrhs)]
    L = _levels(nx)
    if L_exact is None:
        L_exact = max(L - 2, 0)
    return Problem(nx=nx, N=N, kappa=kappa, eta=kappa, bumps=[Bump(amp, cx, cy, 160.0)],
                   thetas=thetas, L_exact=L_exact, inner_iters=inner_iters,
                   name=name or f"{nx}x{nx}_N{N}_k{kappa:g}")


def fp64_64x64(seed: int = 1, nrhs: int = 16) -> Problem:
    """64x64 elements, N=16, kappa=100, one seeded bump, 16 plane waves, L_exact=L-2."""
    return single_bump(64, 16, 100.0, nrhs, seed, L_exact=10, inner_iters=5,
                       name="64x64_N16_k100")


def multi_bump(nx: int, N: int, kappa: float, nbumps: int, nrhs: int, seed: int,
               L_exact: int | None = None, inner_iters: int = 5, name: str = "") -> Problem:
    """Sum of bumps: amplitude U[0,1], width sigma U[0.02,0.1] in exp(-|x-c|^2/(2 sigma^2)),
    centres U[0,1]^2."""
    rng = SplitMix64(seed)
    bumps = []
    for _ in range(nbumps):
        amp = rng.uniform(0.0, 1.0)
        sigma = rng.uniform(0.02, 0.1)
        cx = rng.uniform(0.0, 1.0)
        cy = rng.uniform(0.0, 1.0)
        bumps.append(Bump(amp, cx, cy, 1.0 / (2.0 * sigma * sigma)))
    thetas = [rng.uniform(0.0, 2.0 * math.pi) for _ in range(nrhs)]
    L = _levels(nx)
    if L_exact is None:
        L_exact = max(L - 2, 0)
    return Problem(nx=nx, N=N, kappa=kappa, eta=kappa, bumps=bumps, thetas=thetas,
                   L_exact=L_exact, inner_iters=inner_iters,
                   name=name or f"{nx}x{nx}_N{N}_k{kappa:g}_{nbumps}bumps")


def mixed_128x128(seed: int = 2, nrhs: int = 32) -> Problem:
    """128x128 elements, N=16, kappa=200, 8 seeded bumps, 32 plane waves, L_exact=L-2."""
    return multi_bump(128, 16, 200.0, 8, nrhs, seed, L_exact=12, inner_iters=5,
                      name="128x128_N16_k200")


def batch_mix(count: int = 512, seed: int = 3, grids=(8, 16, 32, 64), orders=(8, 12, 16),
              kappa_range=(20.0, 150.0), rhs_range=(1, 8)) -> list:
    """Independent problems: grid U{grids}, N U{orders}, kappa U[range], 1-8 RHS, one bump."""
    rng = SplitMix64(seed)
    out = []
    for i in range(count):
        nx = rng.choice(list(grids))
        N = rng.choice(list(orders))
        kappa = rng.uniform(*kappa_range)
        nrhs = rng.randint(*rhs_range)
        sub_seed = rng.next_u64()
        p = single_bump(nx, N, kappa, nrhs, sub_seed, name=f"batch{i}")
        out.append(p)
    return out
