"""Pins of the oracle's GMRES / FGMRES (section 4.3) and solver agreement."""
import numpy as np
import pytest

from oracle.krylov import fgmres, gmres_fixed
from oracle.problem import OracleProblem
from oracle.skeleton import assemble_M
from paper_2511_00735_gb300 import inputs


def test_gmres_full_dimension_is_exact():
    rng = np.random.default_rng(0)
    n = 12
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 4 * np.eye(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x = gmres_fixed(lambda v: A @ v, b, n)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-10)


def test_gmres_one_step_closed_form():
    # one step: x = alpha b with alpha = <Ab, b> / <Ab, Ab>
    rng = np.random.default_rng(1)
    A = rng.standard_normal((6, 6)) + 1j * rng.standard_normal((6, 6))
    b = rng.standard_normal(6) + 0j
    Ab = A @ b
    alpha = np.vdot(Ab, b) / np.vdot(Ab, Ab)
    np.testing.assert_allclose(gmres_fixed(lambda v: A @ v, b, 1), alpha * b, rtol=1e-12)


def test_gmres_minimises_residual_over_krylov_space():
    rng = np.random.default_rng(2)
    n, k = 20, 4
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 3 * np.eye(n)
    b = rng.standard_normal(n) + 0j
    x = gmres_fixed(lambda v: A @ v, b, k)
    K = np.stack([np.linalg.matrix_power(A, j) @ b for j in range(k)], axis=1)
    y = np.linalg.lstsq(A @ K, b, rcond=None)[0]
    np.testing.assert_allclose(x, K @ y, rtol=1e-8)


def test_gmres_happy_breakdown():
    A = np.diag([2.0, 2.0, 2.0]) + 0j
    b = np.array([1.0, 1.0, 0.0]) + 0j
    np.testing.assert_allclose(gmres_fixed(lambda v: A @ v, b, 3), b / 2, rtol=1e-14)


def test_fgmres_restart_and_identity_preconditioner():
    rng = np.random.default_rng(3)
    n = 40
    A = np.eye(n) + 0.3 * rng.standard_normal((n, n)) / np.sqrt(n) + 0j
    b = rng.standard_normal(n) + 0j
    x, info = fgmres(lambda v: A @ v, b, None, tol=1e-12, restart=5, max_outer=50)
    assert info["converged"] and info["true_rel_residual"] < 1e-11
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9)


@pytest.fixture(scope="module")
def cfg():
    op = OracleProblem(inputs.small_4x4(0))
    return op


def test_solvers_agree(cfg):
    op = cfg
    g_ref = np.linalg.solve(assemble_M(op.mesh, op.Ts), op.rhs[0])
    g_dir = op.solve_direct()[0]
    g_un, i_un = op.solve_unpreconditioned(tol=1e-10)
    g_mg, i_mg = op.solve_fgmres(L_exact=2, inner_iters=5, tol=1e-10)
    g_ex, i_ex = op.solve_fgmres(L_exact=3, tol=1e-10, coarse="exact")
    for g in (g_dir, g_un[0], g_mg[0], g_ex[0]):
        assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < 1e-8
    assert i_ex[0]["iterations"] == 1
    assert i_mg[0]["iterations"] < i_un[0]["iterations"]
    assert i_mg[0]["true_rel_residual"] < 1e-10


def test_table1_trends(cfg):
    # Table 1: iterations do not increase with more exact levels or more coarse iterations
    op = cfg
    its_L = [op.solve_fgmres(L_exact=L, inner_iters=4, tol=1e-10)[1][0]["iterations"]
             for L in range(0, 4)]
    assert all(b <= a for a, b in zip(its_L, its_L[1:])), its_L
    its_c = [op.solve_fgmres(L_exact=1, inner_iters=c, tol=1e-10)[1][0]["iterations"]
             for c in (2, 4, 8)]
    assert all(b <= a for a, b in zip(its_c, its_c[1:])), its_c


def test_table1_gamma_trend(cfg):
    # Table 1, gamma = 2 columns: with the same coarse steps, two coarse calls per level take
    # no more FGMRES iterations than one (parity unpinned in absolute counts)
    op = cfg
    for L_exact, ci in ((1, 2), (2, 2), (2, 3)):
        it1 = op.solve_fgmres(L_exact=L_exact, inner_iters=ci, tol=1e-10, gamma=1)[1][0]["iterations"]
        it2 = op.solve_fgmres(L_exact=L_exact, inner_iters=ci, tol=1e-10, gamma=2)[1][0]["iterations"]
        assert it2 <= it1, (L_exact, ci, it1, it2)
