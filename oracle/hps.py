"""Nested-dissection merges, direct HPS and the multigrid preconditioner (paper section 4).

Subdomains.  After k merges a subdomain is a block of a x b elements,
a = 2^ceil(k/2), b = 2^floor(k/2) (x-merges at odd levels, y-merges at even
levels, Fig. 1 and reading A14).  Its boundary is numbered in the natural order
l, r, b, t (side lengths bq, bq, aq, aq), each side by increasing coordinate;
position p carries (element, element side, node).  For each position the
oracle keeps the global skeleton unknown incoming to the subdomain there
(`inn`, -1 on the physical boundary), the unknown incoming to the neighbour
across it (`out`), and the physical-boundary data index (`bdr`).

Local merge (eqs. localfacesystem and globalfacesystem).  Subdomain s1 (left /
bottom) and s2 (right / top) share the interface alpha (side of s1) / beta
(side of s2); E1, E2 are their other positions.  With the transmission
reading A3, x = [in2_beta ; in1_alpha] (the paper's ordering) satisfies
    A x = -(B y + h),   A = [[I, T1_aa], [T2_bb, I]],  B = diag(T1_aE1, T2_bE2),
    h = [H1_a ; H2_b],  y = [in1_E1 ; in2_E2],
and the outgoing data on E is C x + D y + [H1_E1; H2_E2] with
    C = [[0, T1_E1a], [T2_E2b, 0]]  (columns follow x's ordering),
    D = diag(T1_E1E1, T2_E2E2).
Hence (reading A4, signs consistent with A3)
    T_pair = D - C A^{-1} B,    H_pair = H_E - C A^{-1} h.
The paper prints C as block diagonal; with x ordered [in2_beta; in1_alpha]
its blocks sit off the diagonal (the product C x is the same).

Multigrid (section 4.3, block-inverse identity):
    MG(M) r = F r + P MG(S) R (I - M F) r,  F = diag(A^{-1}, 0),
    P = [-A^{-1} B ; I],  R = [0 I],  S = D - C A^{-1} B,
one coarse call per level (V-cycle); the coarse system after L_exact merges is
solved by a fixed number of unpreconditioned GMRES steps or exactly.
gamma-cycle (section 4.3, "multiple [coarse calls] define a gamma-cycle";
reading A17): the coarse correction e for S r_c is made by gamma calls, each
on the current residual,
    e_0 = 0,  e_k = e_{k-1} + MG(S) (r_c - S e_{k-1}),  k = 1..gamma,
at every level, the coarsest included (there MG(S) is the coarse solver);
gamma = 1 is the V-cycle.
`mg_dense` applies this formula literally to an assembled M; `MergeTree.mg`
applies the same operator through the per-pair blocks (pinned to `mg_dense`).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .krylov import gmres_fixed
from .skeleton import Mesh, OPP


class Sub:
    """A rectangular subdomain of a x b elements with origin element (ix0, iy0)."""

    def __init__(self, mesh: Mesh, ix0: int, iy0: int, a: int, b: int):
        self.ix0, self.iy0, self.a, self.b = ix0, iy0, a, b
        q = mesh.q
        pos = []
        for t in range(b):
            pos += [(mesh.elem(ix0, iy0 + t), 0, k) for k in range(q)]
        for t in range(b):
            pos += [(mesh.elem(ix0 + a - 1, iy0 + t), 1, k) for k in range(q)]
        for t in range(a):
            pos += [(mesh.elem(ix0 + t, iy0), 2, k) for k in range(q)]
        for t in range(a):
            pos += [(mesh.elem(ix0 + t, iy0 + b - 1), 3, k) for k in range(q)]
        self.pos = pos
        self.n = len(pos)
        self.side = {0: np.arange(0, b * q), 1: np.arange(b * q, 2 * b * q),
                     2: np.arange(2 * b * q, 2 * b * q + a * q),
                     3: np.arange(2 * b * q + a * q, 2 * (a + b) * q)}
        self.inn = np.array([mesh.unknown_in[e, s] + k if mesh.unknown_in[e, s] >= 0 else -1
                             for (e, s, k) in pos], dtype=np.int64)
        self.out = np.array([mesh.unknown_out(e, s) + k if mesh.unknown_out(e, s) >= 0 else -1
                             for (e, s, k) in pos], dtype=np.int64)
        self.bdr = np.array([mesh.bdry_in[e, s] + k if mesh.bdry_in[e, s] >= 0 else -1
                             for (e, s, k) in pos], dtype=np.int64)
        self.T = None
        self.H = None


class MergeRecord:
    """Blocks of one local merge, kept for the sweeps of the preconditioner."""

    def __init__(self, s1: Sub, s2: Sub, ia, ib, E1, E2, A, B, C, keep_blocks=True):
        self.s1, self.s2 = s1, s2
        self.ia, self.ib, self.E1, self.E2 = ia, ib, E1, E2
        self.m = len(ia)
        self.lu = sla.lu_factor(A)
        if keep_blocks:
            self.A, self.B, self.C = A, B, C
        else:
            self.A = None
            self.B, self.C = B, C
        # global unknown indices of x = [in2_beta ; in1_alpha] and of y / rows of C
        self.x_idx = np.concatenate([s2.inn[ib], s1.inn[ia]])
        self.y_inn = np.concatenate([s1.inn[E1], s2.inn[E2]])
        self.y_out = np.concatenate([s1.out[E1], s2.out[E2]])

    def solveA(self, v):
        return sla.lu_solve(self.lu, v)


def merge_pair(mesh: Mesh, s1: Sub, s2: Sub, direction: str, keep_blocks=True):
    """Merge s1 (left/bottom) and s2 (right/top) into one subdomain (eq. globalfacesystem)."""
    if direction == "x":
        alpha, beta = 1, 0
        merged = Sub(mesh, s1.ix0, s1.iy0, s1.a + s2.a, s1.b)
    else:
        alpha, beta = 3, 2
        merged = Sub(mesh, s1.ix0, s1.iy0, s1.a, s1.b + s2.b)
    ia, ib = s1.side[alpha], s2.side[beta]
    E1 = np.array([p for p in range(s1.n) if p not in set(ia.tolist())], dtype=np.int64)
    E2 = np.array([p for p in range(s2.n) if p not in set(ib.tolist())], dtype=np.int64)
    m = len(ia)
    T1, T2 = s1.T, s2.T
    I = np.eye(m)
    A = np.block([[I, T1[np.ix_(ia, ia)]], [T2[np.ix_(ib, ib)], I]])
    Z1 = np.zeros((m, len(E2)))
    Z2 = np.zeros((m, len(E1)))
    B = np.block([[T1[np.ix_(ia, E1)], Z1], [Z2, T2[np.ix_(ib, E2)]]])
    C = np.block([[np.zeros((len(E1), m)), T1[np.ix_(E1, ia)]],
                  [T2[np.ix_(E2, ib)], np.zeros((len(E2), m))]])
    D = np.block([[T1[np.ix_(E1, E1)], np.zeros((len(E1), len(E2)))],
                  [np.zeros((len(E2), len(E1))), T2[np.ix_(E2, E2)]]])
    rec = MergeRecord(s1, s2, ia, ib, E1, E2, A, B, C, keep_blocks)
    Tp = D - C @ rec.solveA(B)
    Hp = None
    if s1.H is not None and s2.H is not None:
        h = np.concatenate([s1.H[ia], s2.H[ib]])
        HE = np.concatenate([s1.H[E1], s2.H[E2]])
        Hp = HE - C @ rec.solveA(h)
    # reorder [E1; E2] into the merged subdomain's natural order
    key = {p: i for i, p in enumerate([s1.pos[k] for k in E1] + [s2.pos[k] for k in E2])}
    perm = np.array([key[p] for p in merged.pos], dtype=np.int64)
    merged.T = Tp[np.ix_(perm, perm)]
    merged.H = Hp[perm] if Hp is not None else None
    return merged, rec


class MergeTree:
    """Stages 0..L_done of the nested-dissection hierarchy (section 4.2)."""

    def __init__(self, mesh: Mesh, Ts, Hs=None, L_exact=None, keep_blocks=True):
        self.mesh = mesh
        L = mesh.L
        if L_exact is None:
            L_exact = L
        if not 0 <= L_exact <= L:
            raise ValueError("0 <= L_exact <= L")
        self.L_exact = L_exact
        leaves = []
        for iy in range(mesh.ny):
            for ix in range(mesh.nx):
                s = Sub(mesh, ix, iy, 1, 1)
                s.T = np.asarray(Ts[mesh.elem(ix, iy)])
                s.H = None if Hs is None else np.asarray(Hs[mesh.elem(ix, iy)])
                leaves.append(s)
        self.stages = [leaves]
        self.grid = [(mesh.nx, mesh.ny)]
        self.merges = [None]
        for lev in range(1, L_exact + 1):
            gx, gy = self.grid[-1]
            cur = self.stages[-1]
            nxt, recs = [], []
            if lev % 2 == 1:
                for j in range(gy):
                    for p in range(gx // 2):
                        s, r = merge_pair(mesh, cur[2 * p + gx * j], cur[2 * p + 1 + gx * j], "x",
                                          keep_blocks)
                        nxt.append(s)
                        recs.append(r)
                self.grid.append((gx // 2, gy))
            else:
                for p in range(gy // 2):
                    for i in range(gx):
                        s, r = merge_pair(mesh, cur[i + gx * (2 * p)], cur[i + gx * (2 * p + 1)], "y",
                                          keep_blocks)
                        nxt.append(s)
                        recs.append(r)
                self.grid.append((gx, gy // 2))
            self.stages.append(nxt)
            self.merges.append(recs)

    # ---- coarse system M_{L_exact+1} ---------------------------------------
    def coarse_index(self) -> np.ndarray:
        idx = np.concatenate([s.inn[s.inn >= 0] for s in self.stages[self.L_exact]])
        return np.sort(idx)

    def coarse_apply(self, g_c, cidx):
        """(M_c g)_u = g_u + (T_c g)_{pi(u)} on the coarse unknowns (global ordering cidx)."""
        n = self.mesh.n_skel
        g = np.zeros((n,) + g_c.shape[1:], dtype=np.complex128)
        g[cidx] = g_c
        out = g.copy()
        for s in self.stages[self.L_exact]:
            gs = np.zeros((s.n,) + g_c.shape[1:], dtype=np.complex128)
            m = s.inn >= 0
            gs[m] = g[s.inn[m]]
            w = s.T @ gs
            mo = s.out >= 0
            out[s.out[mo]] += w[mo]
        return out[cidx]

    def coarse_dense(self, cidx):
        nc = len(cidx)
        return self.coarse_apply(np.eye(nc, dtype=np.complex128), cidx)

    # ---- the system of any stage: M_{k+1} on the unknowns left after k merges ----
    def stage_index(self, k: int) -> np.ndarray:
        idx = np.concatenate([s.inn[s.inn >= 0] for s in self.stages[k]])
        return np.sort(idx)

    def stage_apply(self, k: int, g):
        """M_{k+1} g for a full-length skeleton vector g supported on the stage-k unknowns:
        (M_{k+1} g)_u = g_u + (T_s g_s)_{pi(u)} with the stage-k subdomain maps T_s; the
        result is full length, zero off the stage-k unknowns."""
        g = np.asarray(g, dtype=np.complex128)
        idx = self.stage_index(k)
        out = np.zeros_like(g)
        out[idx] = g[idx]
        for s in self.stages[k]:
            gs = np.zeros(s.n, dtype=np.complex128)
            m = s.inn >= 0
            gs[m] = g[s.inn[m]]
            w = s.T @ gs
            mo = s.out >= 0
            out[s.out[mo]] += w[mo]
        return out

    # ---- the preconditioner ------------------------------------------------
    def mg(self, r, coarse="gmres", inner_iters=5, gamma=1):
        """z = MG(M) r through the per-pair blocks (V-cycle, section 4.3; gamma > 1: the
        gamma-cycle, see mg_gamma)."""
        if gamma != 1:
            return self.mg_gamma(r, coarse, inner_iters, gamma)
        r = np.array(r, dtype=np.complex128)
        zs = []
        for lev in range(1, self.L_exact + 1):
            zl = []
            for rec in self.merges[lev]:
                z = rec.solveA(r[rec.x_idx])                      # F r on this block
                Cz = rec.C @ z
                m = rec.y_out >= 0
                r[rec.y_out[m]] -= Cz[m]                          # R (I - M F) r
                zl.append(z)
            zs.append(zl)
        cidx = self.coarse_index()
        sol = np.zeros_like(r)
        if len(cidx):
            rc = r[cidx]
            if coarse == "exact":
                ec = np.linalg.solve(self.coarse_dense(cidx), rc)
            else:
                ec = gmres_fixed(lambda v: self.coarse_apply(v, cidx), rc, inner_iters)
            sol[cidx] = ec
        for lev in range(self.L_exact, 0, -1):
            for rec, z in zip(self.merges[lev], zs[lev - 1]):
                y = np.zeros(len(rec.y_inn), dtype=np.complex128)
                m = rec.y_inn >= 0
                y[m] = sol[rec.y_inn[m]]
                sol[rec.x_idx] = z - rec.solveA(rec.B @ y)      # P e
        return sol

    def mg_gamma(self, r, coarse="gmres", inner_iters=5, gamma=2):
        """z = MG(M) r with gamma coarse calls per level (section 4.3, reading A17): at level l
        the smoother and restriction of the V-cycle, then e_k = e_{k-1} + MG(M_{l+1})(r_c -
        M_{l+1} e_{k-1}) for k = 1..gamma (MG of the coarsest system = the coarse solver),
        then the prolongation."""
        cidx = self.coarse_index()

        def level(lev, r):
            # MG of M_lev (its unknowns: those of stage lev-1) applied to r
            if lev > self.L_exact:
                sol = np.zeros_like(r)
                if len(cidx):
                    rc = r[cidx]
                    if coarse == "exact":
                        sol[cidx] = np.linalg.solve(self.coarse_dense(cidx), rc)
                    else:
                        sol[cidx] = gmres_fixed(lambda v: self.coarse_apply(v, cidx), rc, inner_iters)
                return sol
            r = r.copy()
            zs = []
            for rec in self.merges[lev]:
                z = rec.solveA(r[rec.x_idx])                      # F r on this block
                Cz = rec.C @ z
                m = rec.y_out >= 0
                r[rec.y_out[m]] -= Cz[m]                          # R (I - M F) r
                zs.append(z)
            idx = self.stage_index(lev)
            rc = np.zeros_like(r)
            rc[idx] = r[idx]
            e = np.zeros_like(r)
            for k in range(gamma):
                res = rc if k == 0 else rc - self.stage_apply(lev, e)
                e = e + level(lev + 1, res)
            sol = e
            for rec, z in zip(self.merges[lev], zs):
                y = np.zeros(len(rec.y_inn), dtype=np.complex128)
                m = rec.y_inn >= 0
                y[m] = sol[rec.y_inn[m]]
                sol[rec.x_idx] = z - rec.solveA(rec.B @ y)      # P e
            return sol

        return level(1, np.array(r, dtype=np.complex128))

    # ---- direct HPS (all merges, boundary data at the root) ----------------
    def direct_solve(self, t):
        """Classic direct HPS: all L merges, then the downward pass from the root's
        boundary data (section 4.2, associativity of Schur complements)."""
        if self.L_exact != self.mesh.L:
            raise ValueError("direct solve needs all L merges")
        t = np.asarray(t, dtype=np.complex128)
        g = np.zeros(self.mesh.n_skel, dtype=np.complex128)

        def incoming(idx_inn, idx_bdr):
            v = np.zeros(len(idx_inn), dtype=np.complex128)
            m = idx_inn >= 0
            v[m] = g[idx_inn[m]]
            v[~m] = t[idx_bdr[~m]]
            return v

        for lev in range(self.mesh.L, 0, -1):
            for rec in self.merges[lev]:
                s1, s2 = rec.s1, rec.s2
                y = np.concatenate([incoming(s1.inn[rec.E1], s1.bdr[rec.E1]),
                                    incoming(s2.inn[rec.E2], s2.bdr[rec.E2])])
                rhs = rec.B @ y
                if s1.H is not None and s2.H is not None:
                    rhs = rhs + np.concatenate([s1.H[rec.ia], s2.H[rec.ib]])
                g[rec.x_idx] = -rec.solveA(rhs)
        return g


def unknown_levels(mesh: Mesh) -> np.ndarray:
    """Merge level of every skeleton unknown (the level of its face)."""
    lv = np.empty(mesh.n_skel, dtype=np.int64)
    for f in range(mesh.nfaces):
        lv[2 * f * mesh.q:(2 * f + 2) * mesh.q] = mesh.face_level(f)
    return lv


def mg_dense(M, levels, lev, L_exact, r, coarse="gmres", inner_iters=5, gamma=1):
    """MG(M) r = F r + P MG(S) R (I - M F) r applied literally to a dense M whose
    unknowns carry merge levels `levels` (plain definition, small meshes only);
    MG(S) r_c is made by gamma calls on the current residual (gamma-cycle)."""
    r = np.asarray(r, dtype=np.complex128)
    if lev > L_exact:
        if len(r) == 0:
            return r.copy()
        if coarse == "exact":
            return np.linalg.solve(M, r)
        return gmres_fixed(lambda v: M @ v, r, inner_iters)
    xs = np.where(levels == lev)[0]
    rest = np.where(levels > lev)[0]
    A = M[np.ix_(xs, xs)]
    B = M[np.ix_(xs, rest)]
    C = M[np.ix_(rest, xs)]
    D = M[np.ix_(rest, rest)]
    Fr = np.zeros_like(r)
    Fr[xs] = np.linalg.solve(A, r[xs])
    rc = (r - M @ Fr)[rest]
    S = D - C @ np.linalg.solve(A, B)
    e = np.zeros(len(rest), dtype=np.complex128)
    for _ in range(gamma):
        e = e + mg_dense(S, levels[rest], lev + 1, L_exact, rc - S @ e, coarse, inner_iters, gamma)
    z = Fr.copy()
    z[rest] += e
    z[xs] += -np.linalg.solve(A, B @ e)
    return z


def schur_levels(M, levels, upto):
    """M_1 = M, M_{l+1} = D_l - C_l A_l^{-1} B_l for l = 1..upto (section 4.2).
    Returns the list [(M_l, levels_l)]."""
    out = [(M, levels)]
    for lev in range(1, upto + 1):
        xs = np.where(levels == lev)[0]
        rest = np.where(levels > lev)[0]
        A = M[np.ix_(xs, xs)]
        B = M[np.ix_(xs, rest)]
        C = M[np.ix_(rest, xs)]
        D = M[np.ix_(rest, rest)]
        M = D - C @ np.linalg.solve(A, B)
        levels = levels[rest]
        out.append((M, levels))
    return out


__all__ = ["Sub", "MergeRecord", "merge_pair", "MergeTree", "unknown_levels", "mg_dense",
           "schur_levels", "OPP"]
