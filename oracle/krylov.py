"""GMRES with a fixed number of steps and flexible GMRES (paper section 4.3).

The coarse level is solved by "a fixed number of unpreconditioned GMRES
iterations" and the outer solver is flexible GMRES with restart 60 and a zero
initial guess (section 5 and Table 1 notes).  Readings A15/A16:

  * coarse GMRES: x0 = 0, no restart, exactly k Arnoldi steps (stop earlier
    only on a happy breakdown h_{j+1,j} <= 1e-14 ||b||), returning the
    least-squares iterate of the Krylov space;
  * outer FGMRES: right-preconditioned flexible GMRES (Saad 1993), modified
    Gram-Schmidt, stop when ||b - M x||_2 / ||b||_2 <= tol (per right-hand
    side), an explicit residual at exit.

The least-squares problems min ||beta e1 - Hbar y|| are solved with numpy's
lstsq (a library primitive); no Givens bookkeeping is needed for a reference.
"""
from __future__ import annotations

import numpy as np


def gmres_fixed(apply_A, b, k: int, breakdown: float = 1e-14):
    """k steps of unpreconditioned GMRES from x0 = 0 (one right-hand side)."""
    b = np.asarray(b, dtype=np.complex128)
    beta = np.linalg.norm(b)
    if beta == 0.0 or k <= 0:
        return np.zeros_like(b)
    V = [b / beta]
    H = np.zeros((k + 1, k), dtype=np.complex128)
    steps = k
    for j in range(k):
        w = apply_A(V[j])
        for i in range(j + 1):
            H[i, j] = np.vdot(V[i], w)
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        if abs(H[j + 1, j]) <= breakdown * beta:
            steps = j + 1
            break
        V.append(w / H[j + 1, j])
    e1 = np.zeros(steps + 1, dtype=np.complex128)
    e1[0] = beta
    y = np.linalg.lstsq(H[:steps + 1, :steps], e1, rcond=None)[0]
    return np.stack(V[:steps], axis=1) @ y


def fgmres(apply_M, b, precond=None, tol: float = 1e-10, restart: int = 60,
           max_outer: int = 20):
    """Right-preconditioned flexible GMRES from x0 = 0 (one right-hand side).

    Returns (x, info) with info = dict(iterations, history (estimated relative
    residual after each step), true_rel_residual, converged)."""
    b = np.asarray(b, dtype=np.complex128)
    if precond is None:
        def precond(v):
            return v
    bnorm = np.linalg.norm(b)
    x = np.zeros_like(b)
    its, hist = 0, []
    converged = bnorm == 0.0
    for _ in range(max_outer):
        if converged:
            break
        r = b - apply_M(x)
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm:
            converged = True
            break
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        y = None
        for j in range(restart):
            z = precond(V[j])
            Z.append(z)
            w = apply_M(z)
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            e1 = np.zeros(j + 2, dtype=np.complex128)
            e1[0] = beta
            y = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)[0]
            res = np.linalg.norm(e1 - H[:j + 2, :j + 1] @ y)
            its += 1
            hist.append(res / bnorm)
            if res <= tol * bnorm or abs(H[j + 1, j]) <= 1e-300:
                converged = res <= tol * bnorm
                break
            V.append(w / H[j + 1, j])
        x = x + np.stack(Z, axis=1) @ y
        if converged:
            break
    true_res = np.linalg.norm(b - apply_M(x)) / (bnorm if bnorm > 0 else 1.0)
    return x, {"iterations": its, "history": hist, "true_rel_residual": true_res,
               "converged": bool(true_res <= tol * 1.0000001 or converged)}
