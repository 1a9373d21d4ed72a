"""1D Gauss-Lobatto-Legendre rule and operators (paper section 3.1).

The paper uses, per element, the tensor-product GLL grid of order N with
quadrature weights w_i, the mass matrix M = diag(w), the differentiation matrix
D and the stiffness matrix K = D^T M D.  It does not state how the rule is
built; this file uses the textbook construction (Canuto, Hussaini, Quarteroni,
Zang, "Spectral Methods", 2006, section 2.3; Kopriva, "Implementing Spectral
Methods for PDEs", 2009, section 3.2):

  * nodes: -1, +1 and the N-1 roots of P_N' (Legendre polynomial derivative),
    found by Newton's method from the Chebyshev-Gauss-Lobatto points;
  * weights: w_j = 2 / (N (N+1) P_N(x_j)^2);
  * differentiation: D_ij = P_N(x_i) / (P_N(x_j) (x_i - x_j)) for i != j,
    D_00 = -N(N+1)/4, D_NN = +N(N+1)/4, all other diagonal entries 0.

Pinned by tests/test_oracle_gll.py (closed-form nodes and weights for N = 2,
3, 4; exactness of quadrature up to degree 2N-1; exactness of D on degree-N
polynomials; the summation-by-parts identity M D + D^T M = diag(-1, 0..0, 1)).
"""
from __future__ import annotations

import numpy as np


def legendre(N: int, x):
    """P_N(x) and P_{N-1}(x) by Bonnet's recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}."""
    x = np.asarray(x, dtype=np.float64)
    p_prev = np.ones_like(x)
    if N == 0:
        return p_prev, np.zeros_like(x)
    p = x.copy()
    for k in range(1, N):
        p_prev, p = p, ((2 * k + 1) * x * p - k * p_prev) / (k + 1)
    return p, p_prev


def gll_rule(N: int):
    """Nodes x_0 < ... < x_N on [-1, 1] and weights of the order-N GLL rule."""
    if N < 1:
        raise ValueError("N >= 1")
    x = np.empty(N + 1)
    x[0], x[N] = -1.0, 1.0
    for j in range(1, N):
        xj = -np.cos(np.pi * j / N)
        for _ in range(100):
            pN, pNm1 = legendre(N, xj)
            dp = N * (pNm1 - xj * pN) / (1.0 - xj * xj)          # P_N'
            d2p = (2.0 * xj * dp - N * (N + 1) * pN) / (1.0 - xj * xj)  # P_N'' from Legendre's ODE
            dx = dp / d2p
            xj = xj - dx
            if abs(dx) < 1e-16:
                break
        x[j] = xj
    pN, _ = legendre(N, x)
    w = 2.0 / (N * (N + 1) * pN ** 2)
    return x, w


def gll_diff(N: int, x=None):
    """GLL differentiation matrix D (D_ij = d ell_j / dx at x_i)."""
    if x is None:
        x, _ = gll_rule(N)
    pN, _ = legendre(N, x)
    D = np.zeros((N + 1, N + 1))
    for i in range(N + 1):
        for j in range(N + 1):
            if i != j:
                D[i, j] = pN[i] / (pN[j] * (x[i] - x[j]))
    D[0, 0] = -N * (N + 1) / 4.0
    D[N, N] = N * (N + 1) / 4.0
    return D


def element_1d(N: int, h: float):
    """Physical 1D operators on an element of width h: (xi, w, D, M, K).

    The paper does not state the scaling; reading: x = x_e + (xi + 1) h / 2, so
    D = (2/h) D_ref and w = (h/2) w_ref, K = D^T M D.
    """
    xi, w_ref = gll_rule(N)
    D = (2.0 / h) * gll_diff(N, xi)
    w = (h / 2.0) * w_ref
    M = np.diag(w)
    K = D.T @ M @ D
    return xi, w, D, M, K
