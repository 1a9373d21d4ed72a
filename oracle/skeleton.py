"""Mesh, faces and the global skeleton system M g = RHS (paper section 3.2).

Mesh: (0,1)^2 split into nx x ny square elements, element e = ix + nx*iy
(x fastest, as in Fig. 1).  Faces:
  vertical   v(ix, iy), ix = 0..nx-2, between (ix, iy) [side r] and (ix+1, iy) [side l],
             face number ix + (nx-1) iy;
  horizontal h(ix, iy), iy = 0..ny-2, between (ix, iy) [side t] and (ix, iy+1) [side b],
             face number (nx-1) ny + ix + nx iy.
Each face carries 2q unknowns (q = N-1): slot 0 = incoming impedance of the
left/bottom element on its side r/t, slot 1 = incoming impedance of the
right/top element on its side l/b; unknown index (2 f + slot) q + k.

Transmission (eq. before faceequations).  Reading A3: with outward normals
per element, continuity of u and of the flux gives
    (I_i u)^(e2)_beta = - (I_o u)^(e1)_alpha
(the paper prints "+").  The plane-wave test pins the sign.

Row convention: the row for unknown g_k is the outgoing relation (eq. localiti)
of the element on the other side of the face, so M = I + Pi T (identity
diagonal, as in eq. faceequations):
    g_{k} + sum_{beta interior} T^(e)_{alpha beta} g^(e)_beta
        = -( H^(e)_alpha + sum_{beta on boundary} T^(e)_{alpha beta} t^(e)_beta ),
where (e, alpha) is the side across the face from unknown k.

Physical boundary data t is a vector of 4 nx q values: domain sides left
(ix = 0, iy = 0..ny-1), right, bottom (iy = 0, ix = 0..nx-1), top, each element
side with its q edge nodes by increasing coordinate.
"""
from __future__ import annotations

import numpy as np

from .gll import gll_rule
from .leaf import SIDES

OPP = {0: 1, 1: 0, 2: 3, 3: 2}


class Mesh:
    def __init__(self, nx: int, ny: int, N: int):
        if nx != ny:
            raise ValueError("square element grids only (domain (0,1)^2, square elements)")
        self.nx, self.ny, self.N = nx, ny, N
        self.q = N - 1
        self.h = 1.0 / nx
        self.E = nx * ny
        self.nv = (nx - 1) * ny
        self.nh = nx * (ny - 1)
        self.nfaces = self.nv + self.nh
        self.n_skel = 2 * self.nfaces * self.q
        self.n_bdry = 2 * (nx + ny) * self.q
        # faces: (e1, side1, e2, side2)
        self.faces = []
        for iy in range(ny):
            for ix in range(nx - 1):
                self.faces.append((self.elem(ix, iy), 1, self.elem(ix + 1, iy), 0))
        for iy in range(ny - 1):
            for ix in range(nx):
                self.faces.append((self.elem(ix, iy), 3, self.elem(ix, iy + 1), 2))
        # unknown_in[e, side]: first index of the unknowns incoming to e on that side (-1: boundary)
        self.unknown_in = -np.ones((self.E, 4), dtype=np.int64)
        self.nbr = -np.ones((self.E, 4), dtype=np.int64)
        for f, (e1, s1, e2, s2) in enumerate(self.faces):
            self.unknown_in[e1, s1] = (2 * f + 0) * self.q
            self.unknown_in[e2, s2] = (2 * f + 1) * self.q
            self.nbr[e1, s1] = e2
            self.nbr[e2, s2] = e1
        # boundary data index
        self.bdry_in = -np.ones((self.E, 4), dtype=np.int64)
        off = {0: 0, 1: ny, 2: 2 * ny, 3: 2 * ny + nx}
        for iy in range(ny):
            self.bdry_in[self.elem(0, iy), 0] = (off[0] + iy) * self.q
            self.bdry_in[self.elem(nx - 1, iy), 1] = (off[1] + iy) * self.q
        for ix in range(nx):
            self.bdry_in[self.elem(ix, 0), 2] = (off[2] + ix) * self.q
            self.bdry_in[self.elem(ix, ny - 1), 3] = (off[3] + ix) * self.q

    def elem(self, ix: int, iy: int) -> int:
        return ix + self.nx * iy

    def coords(self, e: int):
        return e % self.nx, e // self.nx

    def unknown_out(self, e: int, side: int) -> int:
        """First index of the unknowns incoming to the neighbour across (e, side)."""
        nb = self.nbr[e, side]
        if nb < 0:
            return -1
        return int(self.unknown_in[nb, OPP[side]])

    # ---- geometry -------------------------------------------------------
    def node_xy(self, e: int):
        """Physical coordinates of the (N+1)^2 nodes of element e, node(i,j) = i(N+1)+j."""
        xi, _ = gll_rule(self.N)
        ix, iy = self.coords(e)
        xs = ix * self.h + (xi + 1.0) * self.h / 2.0
        ys = iy * self.h + (xi + 1.0) * self.h / 2.0
        X = np.repeat(xs, self.N + 1)
        Y = np.tile(ys, self.N + 1)
        return X, Y

    def all_node_xy(self):
        X = np.empty((self.E, (self.N + 1) ** 2))
        Y = np.empty_like(X)
        for e in range(self.E):
            X[e], Y[e] = self.node_xy(e)
        return X, Y

    def side_xy(self, e: int, side: int):
        """Coordinates and outward normal of the q edge nodes on a side of element e."""
        xi, _ = gll_rule(self.N)
        ix, iy = self.coords(e)
        x0, y0 = ix * self.h, iy * self.h
        t = (xi[1:-1] + 1.0) * self.h / 2.0
        if side == 0:
            return np.full(self.q, x0), y0 + t, (-1.0, 0.0)
        if side == 1:
            return np.full(self.q, x0 + self.h), y0 + t, (1.0, 0.0)
        if side == 2:
            return x0 + t, np.full(self.q, y0), (0.0, -1.0)
        return x0 + t, np.full(self.q, y0 + self.h), (0.0, 1.0)

    def boundary_points(self):
        """Coordinates and normals of the n_bdry physical boundary nodes (t-vector order)."""
        X = np.empty(self.n_bdry)
        Y = np.empty(self.n_bdry)
        NX = np.empty(self.n_bdry)
        NY = np.empty(self.n_bdry)
        for e in range(self.E):
            for s in range(4):
                b = self.bdry_in[e, s]
                if b >= 0:
                    x, y, n = self.side_xy(e, s)
                    X[b:b + self.q], Y[b:b + self.q] = x, y
                    NX[b:b + self.q], NY[b:b + self.q] = n
        return X, Y, NX, NY

    # ---- nested-dissection levels (section 4.2, Fig. 1) -------------------
    @property
    def L(self) -> int:
        k = int(round(np.log2(self.nx)))
        return 2 * k

    def face_level(self, f: int) -> int:
        """Merge level that eliminates face f: x-merges at odd levels, y-merges at even
        levels; a cut at grid line p is removed at the level where the subdomain
        width (height) first reaches past it."""
        e1, s1, _, _ = self.faces[f]
        ix, iy = self.coords(e1)
        if s1 == 1:
            p = ix + 1
            return 2 * _v2(p) + 1
        p = iy + 1
        return 2 * (_v2(p) + 1)


def _v2(p: int) -> int:
    k = 0
    while p % 2 == 0:
        p //= 2
        k += 1
    return k


def side_slice(q: int, side: int) -> slice:
    return slice(side * q, (side + 1) * q)


def assemble_M(mesh: Mesh, Ts) -> np.ndarray:
    """Dense skeleton matrix M (n_skel x n_skel), rows as in the module docstring."""
    q = mesh.q
    M = np.eye(mesh.n_skel, dtype=np.complex128)
    for e in range(mesh.E):
        for a in range(4):
            row = mesh.unknown_out(e, a)
            if row < 0:
                continue
            for b in range(4):
                col = mesh.unknown_in[e, b]
                if col < 0:
                    continue
                M[row:row + q, col:col + q] += Ts[e][side_slice(q, a), side_slice(q, b)]
    return M


def assemble_rhs(mesh: Mesh, Ts, t, Hs=None) -> np.ndarray:
    """RHS_k = -(H^(e)_alpha + sum_{beta on boundary} T^(e)_{alpha beta} t_beta)."""
    q = mesh.q
    t = np.asarray(t, dtype=np.complex128)
    rhs = np.zeros(mesh.n_skel, dtype=np.complex128)
    for e in range(mesh.E):
        for a in range(4):
            row = mesh.unknown_out(e, a)
            if row < 0:
                continue
            acc = np.zeros(q, dtype=np.complex128)
            if Hs is not None:
                acc += Hs[e][side_slice(q, a)]
            for b in range(4):
                bi = mesh.bdry_in[e, b]
                if bi >= 0:
                    acc += Ts[e][side_slice(q, a), side_slice(q, b)] @ t[bi:bi + q]
            rhs[row:row + q] = -acc
    return rhs


def apply_M(mesh: Mesh, Ts, g) -> np.ndarray:
    """M g without assembling M (same rows as assemble_M); g may be (n_skel,) or (n_skel, k)."""
    q = mesh.q
    g = np.asarray(g, dtype=np.complex128)
    out = g.copy()
    for e in range(mesh.E):
        ge = np.zeros((4 * q,) + g.shape[1:], dtype=np.complex128)
        for b in range(4):
            col = mesh.unknown_in[e, b]
            if col >= 0:
                ge[side_slice(q, b)] = g[col:col + q]
        w = Ts[e] @ ge
        for a in range(4):
            row = mesh.unknown_out(e, a)
            if row >= 0:
                out[row:row + q] += w[side_slice(q, a)]
    return out


def element_incoming(mesh: Mesh, g, t, e: int) -> np.ndarray:
    """Incoming impedance data of element e on iota_Gamma from the skeleton g and boundary t."""
    q = mesh.q
    f = np.zeros(4 * q, dtype=np.complex128)
    for s in range(4):
        u = mesh.unknown_in[e, s]
        if u >= 0:
            f[side_slice(q, s)] = g[u:u + q]
        else:
            b = mesh.bdry_in[e, s]
            f[side_slice(q, s)] = t[b:b + q]
    return f


def volume_system(mesh: Mesh, cs, eta: float, t):
    """Brute-force global volume system (independent of the skeleton reduction).

    Unknowns: all (N+1)^2 nodes of every element (edge nodes duplicated).
    Rows per element: corners u = 0; interior nodes L~(iota_i, :) u = 0;
    edge nodes on the physical boundary I_i u = t; edge nodes on an interior
    face I_i^(e) u^(e) + I_o^(nbr) u^(nbr) = 0 (reading A3), matching nodes of
    the two sides index for index.  Returns (A, rhs).
    """
    from .leaf import element_operators, index_sets

    N, q = mesh.N, mesh.q
    n = (N + 1) ** 2
    ops = [element_operators(N, mesh.h, cs[e], eta) for e in range(mesh.E)]
    s = index_sets(N)
    A = np.zeros((mesh.E * n, mesh.E * n), dtype=np.complex128)
    rhs = np.zeros(mesh.E * n, dtype=np.complex128)
    for e in range(mesh.E):
        Lt, Dn, Ii, Io, _ = ops[e]
        base = e * n
        for cn in s["corners"]:
            A[base + cn, base + cn] = 1.0
        for k in s["interior"]:
            A[base + k, base:base + n] = Lt[k]
        for side in range(4):
            rows_g = range(side * q, (side + 1) * q)
            nodes = s[SIDES[side]]
            nb = mesh.nbr[e, side]
            for kk, (rg, nd) in enumerate(zip(rows_g, nodes)):
                A[base + nd, base:base + n] = Ii[rg]
                if nb < 0:
                    b = mesh.bdry_in[e, side]
                    rhs[base + nd] = t[b + kk]
                else:
                    _, _, _, Io_nb, _ = ops[nb]
                    rg_nb = OPP[side] * q + kk
                    A[base + nd, nb * n:(nb + 1) * n] += Io_nb[rg_nb]
    return A, rhs
