"""Leaf (element) impedance-to-impedance map (paper section 3.1, eq. ItIOperator).

Per element, with tensor GLL nodes (x_i, y_j), i, j = 0..N, numbered
node(i, j) = i (N+1) + j (x index slow, so that D_x (x) I is kron(D, I)):

  L~ = K_x (x) M_y + M_x (x) K_y - diag(c(x_i, y_j)) (M_x (x) M_y),   c = kappa^2 (1 - b)

  Reading A1: the paper prints "+ diag(c)"; the PDE -Lap u - c u = s has weak
  form (grad u, grad v) - (c u, v), so the sign used here is "-".  The
  plane-wave test (tests/test_oracle_leaf.py, test_oracle_global.py) fails
  with "+".

  Outgoing / incoming impedance operators on the edge (non-corner) nodes
  iota_Gamma = [iota_l, iota_r, iota_b, iota_t]:
      Dn = [ -D_x(x)I ; D_x(x)I ; -I(x)D_y ; I(x)D_y ](iota_Gamma, :)   (outward normal derivative)
      I_o = Dn - i eta I(iota_Gamma, :),  I_i = Dn + i eta I(iota_Gamma, :)
  Reading A2: the paper prints "-eta I" / "+eta I" without the imaginary unit;
  the boundary condition du/dn + i eta u = t requires i eta.

  L(iota_Gamma, :) = I_i, L(iota_i, :) = L~(iota_i, :); the four corner nodes
  are removed (or, equivalently, given identity rows: no other row touches a
  corner column, so both layouts give the same T -- pinned).

  T = I_o L^{-1} I(:, iota_Gamma),   H = I_o L^{-1} I(:, iota_i) b~(iota_i).

  Reading A7: b~(iota_i) = w_i w_j s(x_i, y_j): the interior rows of L~ equal
  w_i w_j (-Lap - c) at the node by the GLL summation-by-parts property
  (pinned by the manufactured-solution test).

Side order l, r, b, t; along a side, nodes by increasing coordinate.
"""
from __future__ import annotations

import numpy as np

from .gll import element_1d

SIDES = ("l", "r", "b", "t")


def node(N: int, i: int, j: int) -> int:
    return i * (N + 1) + j


def index_sets(N: int) -> dict:
    """iota_l, iota_r, iota_b, iota_t, iota_Gamma, iota_i and the corners."""
    q = range(1, N)
    s = {
        "l": [node(N, 0, j) for j in q],
        "r": [node(N, N, j) for j in q],
        "b": [node(N, i, 0) for i in q],
        "t": [node(N, i, N) for i in q],
    }
    s["gamma"] = s["l"] + s["r"] + s["b"] + s["t"]
    s["interior"] = [node(N, i, j) for i in q for j in q]
    s["corners"] = [node(N, 0, 0), node(N, 0, N), node(N, N, 0), node(N, N, N)]
    return s


def element_operators(N: int, h: float, c, eta: float):
    """Return (Lt, Dn, Ii, Io, sets) for one element; c holds (N+1)^2 node values."""
    _, w, D, M, K = element_1d(N, h)
    I1 = np.eye(N + 1)
    c = np.asarray(c, dtype=np.float64).reshape(-1)
    Lt = np.kron(K, M) + np.kron(M, K) - np.diag(c) @ np.kron(M, M)
    Dx = np.kron(D, I1)
    Dy = np.kron(I1, D)
    s = index_sets(N)
    Dn = np.vstack([-Dx[s["l"]], Dx[s["r"]], -Dy[s["b"]], Dy[s["t"]]])
    Ig = np.eye((N + 1) ** 2)[s["gamma"]]
    Ii = Dn + 1j * eta * Ig
    Io = Dn - 1j * eta * Ig
    return Lt, Dn, Ii, Io, s


def leaf_matrix(N: int, h: float, c, eta: float, corners: str = "identity"):
    """The element matrix L (complex) and I_o, in the 289-node layout with
    identity corner rows (corners='identity') or with corners removed ('drop').

    Returns (L, Io, keep) where keep lists the retained node indices."""
    Lt, Dn, Ii, Io, s = element_operators(N, h, c, eta)
    n = (N + 1) ** 2
    L = Lt.astype(np.complex128)
    L[s["gamma"], :] = Ii
    for cn in s["corners"]:
        L[cn, :] = 0.0
        L[cn, cn] = 1.0
    keep = list(range(n))
    if corners == "drop":
        keep = [k for k in range(n) if k not in s["corners"]]
        L = L[np.ix_(keep, keep)]
        Io = Io[:, keep]
    return L, Io, keep


def leaf_itI(N: int, h: float, c, eta: float, btilde=None, corners: str = "identity"):
    """Leaf ItI map T (4(N-1) x 4(N-1)) and interior contribution H (eq. ItIOperator).

    btilde: optional (N+1)^2 array of local right-hand-side values (only its
    interior entries are used).  Returns dict(T=..., H=..., Y=...), where
    Y = L^{-1} I(:, iota_Gamma) in the full 289-node numbering.
    """
    s = index_sets(N)
    L, Io, keep = leaf_matrix(N, h, c, eta, corners)
    n = (N + 1) ** 2
    pos = {k: a for a, k in enumerate(keep)}
    E_gamma = np.zeros((len(keep), len(s["gamma"])), dtype=np.complex128)
    for col, k in enumerate(s["gamma"]):
        E_gamma[pos[k], col] = 1.0
    Yk = np.linalg.solve(L, E_gamma)
    T = Io @ Yk
    Y = np.zeros((n, len(s["gamma"])), dtype=np.complex128)
    Y[keep, :] = Yk
    H = np.zeros(len(s["gamma"]), dtype=np.complex128)
    if btilde is not None:
        bt = np.asarray(btilde, dtype=np.complex128).reshape(-1)
        rhs = np.zeros(len(keep), dtype=np.complex128)
        for k in s["interior"]:
            rhs[pos[k]] = bt[k]
        H = Io @ np.linalg.solve(L, rhs)
    return {"T": T, "H": H, "Y": Y}


def leaf_solution(N: int, h: float, c, eta: float, f_in, btilde=None):
    """Element field u from incoming impedance data f_in on iota_Gamma (section 3.1):
    L u = b with b(iota_Gamma) = f_in, b(iota_i) = b~(iota_i); corners returned as 0."""
    s = index_sets(N)
    L, _, _ = leaf_matrix(N, h, c, eta, "identity")
    b = np.zeros((N + 1) ** 2, dtype=np.complex128)
    b[s["gamma"]] = f_in
    if btilde is not None:
        bt = np.asarray(btilde, dtype=np.complex128).reshape(-1)
        b[s["interior"]] = bt[s["interior"]]
    return np.linalg.solve(L, b)


def corner_values(N: int, u):
    """Corner post-processing (section 3.1: the corners are removed from the discretization and
    "recalculated later in post-processing").  Reading: the value at a corner is the mean of the
    two one-sided extrapolations along the element edges that meet there, each the value at the
    edge's end point of the degree N-2 polynomial through that edge's N-1 non-corner nodes.
    Exact for fields whose edge restrictions have degree <= N-2; spectrally accurate for smooth
    fields.  Returns a copy of u (all (N+1)^2 nodes) with the four corners filled."""
    from .gll import gll_rule

    xi, _ = gll_rule(N)
    inner = xi[1:N]

    def end_weights(x_end):
        # Lagrange basis of the interior nodes evaluated at x_end
        w = np.ones(N - 1)
        for j in range(N - 1):
            for k in range(N - 1):
                if k != j:
                    w[j] *= (x_end - inner[k]) / (inner[j] - inner[k])
        return w

    wl, wr = end_weights(-1.0), end_weights(1.0)
    u = np.array(u, dtype=np.complex128).reshape(-1).copy()
    q = range(1, N)
    left = np.array([u[node(N, 0, j)] for j in q])
    right = np.array([u[node(N, N, j)] for j in q])
    bottom = np.array([u[node(N, i, 0)] for i in q])
    top = np.array([u[node(N, i, N)] for i in q])
    u[node(N, 0, 0)] = 0.5 * (wl @ left + wl @ bottom)
    u[node(N, 0, N)] = 0.5 * (wr @ left + wl @ top)
    u[node(N, N, 0)] = 0.5 * (wl @ right + wr @ bottom)
    u[node(N, N, N)] = 0.5 * (wr @ right + wr @ top)
    return u


def interior_weights(N: int, h: float):
    """w_i w_j at every node (used to form b~ = w_i w_j s, reading A7)."""
    _, w, _, _, _ = element_1d(N, h)
    return np.kron(w, w)
