"""Pins of the oracle's skeleton system and direct HPS (sections 3.2, 4.2)."""
import numpy as np
import pytest

from oracle.leaf import corner_values, index_sets, interior_weights, leaf_solution
from oracle.problem import OracleProblem, coefficient
from oracle.skeleton import Mesh, apply_M, assemble_M, element_incoming, volume_system
from paper_2511_00735_gb300 import inputs


def exact_skeleton(mesh, theta, kappa, eta):
    g = np.zeros(mesh.n_skel, dtype=complex)
    for e in range(mesh.E):
        for s in range(4):
            u = mesh.unknown_in[e, s]
            if u >= 0:
                x, y, n = mesh.side_xy(e, s)
                g[u:u + mesh.q] = inputs.plane_wave_impedance(theta, kappa, eta, x, y, *n)
    return g


@pytest.mark.parametrize("N,tol", [(8, 2e-6), (12, 1e-10), (16, 5e-12)])
def test_plane_wave_b0(N, tol):
    p = inputs.Problem(nx=4, N=N, kappa=10.0, eta=10.0, bumps=[], thetas=[0.7])
    op = OracleProblem(p)
    g = np.linalg.solve(assemble_M(op.mesh, op.Ts), op.rhs[0])
    gex = exact_skeleton(op.mesh, 0.7, 10.0, 10.0)
    assert np.linalg.norm(g - gex) / np.linalg.norm(gex) < tol
    # recovered volume field matches the plane wave at all non-corner nodes
    mesh = op.mesh
    c = coefficient(mesh, 10.0, [])
    corners = set(index_sets(N)["corners"])
    errs = []
    for e in range(mesh.E):
        u = leaf_solution(N, mesh.h, c[e], 10.0, element_incoming(mesh, g, op.ts[0], e))
        X, Y = mesh.node_xy(e)
        ue = inputs.plane_wave(0.7, 10.0, X, Y)
        k = [i for i in range(len(u)) if i not in corners]
        errs.append(np.max(abs(u[k] - ue[k])))
    assert max(errs) < 10 * tol


def test_transmission_plus_sign_fails():
    # planted mistake: the printed "+" transmission sign (M = I - Pi T, RHS negated)
    p = inputs.Problem(nx=4, N=12, kappa=10.0, eta=10.0, bumps=[], thetas=[0.7])
    op = OracleProblem(p)
    M = assemble_M(op.mesh, op.Ts)
    Mbad = 2 * np.eye(len(M)) - M
    g = np.linalg.solve(Mbad, -op.rhs[0])
    gex = exact_skeleton(op.mesh, 0.7, 10.0, 10.0)
    assert np.linalg.norm(g - gex) / np.linalg.norm(gex) > 1e-2


def test_manufactured_solution_b_nonzero():
    # s = kappa^2 b u_pw, t = I_i u_pw  =>  u = u_pw (pins the H path and reading A7)
    kappa, theta = 10.0, 1.1
    bumps = [inputs.PAPER_BUMP]
    p = inputs.Problem(nx=4, N=12, kappa=kappa, eta=kappa, bumps=bumps, thetas=[theta])

    def source(X, Y):
        return kappa ** 2 * inputs.eval_b(bumps, X, Y) * inputs.plane_wave(theta, kappa, X, Y)

    op = OracleProblem(p, source=source)
    g = np.linalg.solve(assemble_M(op.mesh, op.Ts), op.rhs[0])
    gex = exact_skeleton(op.mesh, theta, kappa, kappa)
    assert np.linalg.norm(g - gex) / np.linalg.norm(gex) < 1e-7
    gd = op.solve_direct()[0]
    assert np.linalg.norm(gd - g) / np.linalg.norm(g) < 1e-12
    # the volume field with the source (b~ = w_i w_j s) and the corners post-processed equals
    # the plane wave at every node, corners included
    mesh = op.mesh
    c = coefficient(mesh, kappa, bumps)
    w2 = interior_weights(p.N, mesh.h)
    err = 0.0
    for e in range(mesh.E):
        X, Y = mesh.node_xy(e)
        u = leaf_solution(p.N, mesh.h, c[e], kappa, element_incoming(mesh, g, op.ts[0], e), w2 * source(X, Y))
        u = corner_values(p.N, u)
        err = max(err, np.max(np.abs(u - inputs.plane_wave(theta, kappa, X, Y))))
    assert err < 1e-6, err


def test_direct_hps_equals_dense_and_volume_solve():
    p = inputs.small_4x4(0)
    op = OracleProblem(p)
    mesh = op.mesh
    g_dense = np.linalg.solve(assemble_M(mesh, op.Ts), op.rhs[0])
    g_direct = op.solve_direct()[0]
    assert np.linalg.norm(g_direct - g_dense) / np.linalg.norm(g_dense) < 1e-11
    # brute force: global volume system with duplicated edge nodes
    c = coefficient(mesh, p.kappa, p.bumps)
    A, rhs = volume_system(mesh, c, p.eta, op.ts[0])
    u = np.linalg.solve(A, rhs)
    from oracle.leaf import element_operators
    n = (mesh.N + 1) ** 2
    g_vol = np.zeros(mesh.n_skel, dtype=complex)
    for e in range(mesh.E):
        _, _, Ii, _, _ = element_operators(mesh.N, mesh.h, c[e], p.eta)
        fi = Ii @ u[e * n:(e + 1) * n]
        for s in range(4):
            k = mesh.unknown_in[e, s]
            if k >= 0:
                g_vol[k:k + mesh.q] = fi[s * mesh.q:(s + 1) * mesh.q]
    assert np.linalg.norm(g_vol - g_dense) / np.linalg.norm(g_dense) < 1e-11


def test_structured_matvec_equals_dense():
    p = inputs.small_4x4(3)
    op = OracleProblem(p)
    M = assemble_M(op.mesh, op.Ts)
    x = np.random.default_rng(0).standard_normal((op.mesh.n_skel, 3)) * (1 + 1j)
    np.testing.assert_allclose(apply_M(op.mesh, op.Ts, x), M @ x, atol=1e-12)


def test_mesh_counts():
    for nx, N, nf, nu in [(4, 8, 24, 336), (64, 16, 8064, 241920), (128, 16, 32512, 975360)]:
        m = Mesh(nx, nx, N) if nx <= 64 else None
        if m is None:
            assert 2 * nx * (nx - 1) == nf and nf * 2 * (N - 1) == nu
            continue
        assert m.nfaces == nf and m.n_skel == nu
