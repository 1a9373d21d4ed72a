"""End-to-end oracle runs for one scattering problem (sections 2-4).

Builds every leaf from the coefficient c = kappa^2 (1 - b) sampled at the
oracle's own GLL nodes, the plane-wave impedance data t on the physical
boundary, the skeleton RHS, and solves M g = RHS with
  * direct HPS (all merges),
  * FGMRES preconditioned by MG(M) with L_exact exact merges and a coarse
    level solved by `inner_iters` GMRES steps (or exactly),
  * unpreconditioned FGMRES.
"""
from __future__ import annotations

import numpy as np

from paper_2511_00735_gb300 import inputs

from .hps import MergeTree
from .krylov import fgmres
from .leaf import interior_weights, leaf_itI
from .skeleton import Mesh, apply_M, assemble_rhs


def coefficient(mesh: Mesh, kappa: float, bumps):
    """c = kappa^2 (1 - b) at every node of every element, shape (E, (N+1)^2)."""
    X, Y = mesh.all_node_xy()
    return kappa ** 2 * (1.0 - inputs.eval_b(bumps, X, Y))


def build_leaves(mesh: Mesh, kappa: float, eta: float, bumps, source=None, elements=None):
    """Leaf T (and H when a source s(x, y) callable is given) for the listed elements."""
    c = coefficient(mesh, kappa, bumps)
    w2 = interior_weights(mesh.N, mesh.h)
    Ts, Hs = {}, {}
    els = range(mesh.E) if elements is None else elements
    for e in els:
        bt = None
        if source is not None:
            X, Y = mesh.node_xy(e)
            bt = w2 * source(X, Y)
        out = leaf_itI(mesh.N, mesh.h, c[e], eta, btilde=bt)
        Ts[e] = out["T"]
        Hs[e] = out["H"]
    if elements is None:
        return [Ts[e] for e in range(mesh.E)], [Hs[e] for e in range(mesh.E)]
    return Ts, Hs


def plane_wave_data(mesh: Mesh, theta: float, kappa: float, eta: float):
    """Impedance data t = du_pw/dn + i eta u_pw at the physical boundary nodes."""
    X, Y, NX, NY = mesh.boundary_points()
    return inputs.plane_wave_impedance(theta, kappa, eta, X, Y, NX, NY)


class OracleProblem:
    def __init__(self, prob: inputs.Problem, source=None):
        self.prob = prob
        self.mesh = Mesh(prob.nx, prob.ny, prob.N)
        self.Ts, self.Hs = build_leaves(self.mesh, prob.kappa, prob.eta, prob.bumps, source)
        self.has_source = source is not None
        self.ts = [plane_wave_data(self.mesh, th, prob.kappa, prob.eta) for th in prob.thetas]
        Hs = self.Hs if self.has_source else None
        self.rhs = [assemble_rhs(self.mesh, self.Ts, t, Hs) for t in self.ts]

    def matvec(self, g):
        return apply_M(self.mesh, self.Ts, g)

    def tree(self, L_exact):
        Hs = self.Hs if self.has_source else None
        return MergeTree(self.mesh, self.Ts, Hs, L_exact)

    def solve_direct(self):
        tree = self.tree(self.mesh.L)
        return [tree.direct_solve(t) for t in self.ts]

    def solve_fgmres(self, L_exact=None, inner_iters=None, tol=1e-10, coarse="gmres",
                     restart=60, max_outer=20, tree=None, gamma=1):
        L_exact = self.prob.L_exact if L_exact is None else L_exact
        inner_iters = self.prob.inner_iters if inner_iters is None else inner_iters
        if tree is None:
            tree = self.tree(L_exact)
        sols, infos = [], []
        for rhs in self.rhs:
            x, info = fgmres(self.matvec, rhs, lambda v: tree.mg(v, coarse, inner_iters, gamma), tol,
                             restart, max_outer)
            sols.append(x)
            infos.append(info)
        return sols, infos

    def solve_unpreconditioned(self, tol=1e-10, restart=60, max_outer=50):
        sols, infos = [], []
        for rhs in self.rhs:
            x, info = fgmres(self.matvec, rhs, None, tol, restart, max_outer)
            sols.append(x)
            infos.append(info)
        return sols, infos

    def rel_residual(self, g, k=0):
        r = self.rhs[k] - self.matvec(g)
        return np.linalg.norm(r) / np.linalg.norm(self.rhs[k])
