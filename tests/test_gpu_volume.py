"""Sources s != 0 and the volume solution on the GPU against the oracle (section 3.1).

Sources enter the skeleton RHS through the leaf interior contributions H of eq. ItIOperator;
the element fields follow from L u = [I_i u ; b~] with the corners post-processed.  The oracle
side is the dense element solve (oracle.leaf.leaf_solution) with its corner post-processing
(oracle.leaf.corner_values) and the dense skeleton system with H (oracle.problem); the
manufactured solution s = kappa^2 b u_pw, t = I_i u_pw has u = u_pw exactly.
Tolerances: 1e-10 relative for element fields computed from the same skeleton data (FP64
dense solves against the CUDA path's refined interior solves), 1e-8 for solutions of the
skeleton system (its conditioning), discretization error for the plane-wave comparisons.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.leaf import corner_values, interior_weights, leaf_solution
from oracle.problem import OracleProblem, coefficient
from oracle.skeleton import Mesh, assemble_M, element_incoming
from paper_2511_00735_gb300 import hps as H
from paper_2511_00735_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def solver():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    s = H.Solver(0)
    yield s
    s.close()


def manufactured(kappa, bumps):
    def source_of(theta):
        return lambda X, Y: kappa ** 2 * inputs.eval_b(bumps, X, Y) * inputs.plane_wave(theta, kappa, X, Y)
    return source_of


def sources(solver, fns):
    X, Y = solver.node_coords()
    return np.ascontiguousarray(np.stack([f(X, Y) for f in fns]).astype(np.complex128))


def oracle_fields(op, g, t, fns):
    """Oracle element fields (all nodes, corners post-processed) for skeleton data g."""
    mesh, N = op.mesh, op.prob.N
    c = coefficient(mesh, op.prob.kappa, op.prob.bumps)
    w2 = interior_weights(N, mesh.h)
    out = []
    for k, fn in enumerate(fns):
        rows = []
        for e in range(mesh.E):
            X, Y = mesh.node_xy(e)
            bt = None if fn is None else w2 * fn(X, Y)
            u = leaf_solution(N, mesh.h, c[e], op.prob.eta, element_incoming(mesh, g[k], t[k], e), bt)
            rows.append(corner_values(N, u))
        out.append(np.stack(rows))
    return np.stack(out)


@pytest.mark.parametrize("nx,N,kappa", [(4, 12, 10.0), (8, 8, 150.0), (8, 8, 36.0)])
def test_source_rhs_solve_and_volume_vs_oracle(solver, nx, N, kappa):
    """(4, 12, 10): every element on the positive-definite route; (8, 8, 150): every element on
    the pivoted route; (8, 8, 36): both."""
    bumps = [inputs.PAPER_BUMP]
    thetas = [0.4, 2.2]
    prob = inputs.Problem(nx=nx, N=N, kappa=kappa, eta=kappa, bumps=bumps, thetas=thetas, L_exact=2)
    fns = [manufactured(kappa, bumps)(th) for th in thetas]
    op = OracleProblem(inputs.Problem(nx=nx, N=N, kappa=kappa, eta=kappa, bumps=bumps, thetas=[thetas[0]]),
                       source=fns[0])
    op2 = OracleProblem(inputs.Problem(nx=nx, N=N, kappa=kappa, eta=kappa, bumps=bumps, thetas=[thetas[1]]),
                        source=fns[1])
    t = H.setup(solver, prob, H.HPS_FP64)
    s = sources(solver, fns)
    solver.merge_levels(prob.L_exact)
    g, info = solver.gmres_solve(t, tol=1e-10, inner_iters=5, max_outer=40, s=s)
    assert info["converged"] == 2
    M = assemble_M(op.mesh, op.Ts)
    g_ref = [np.linalg.solve(M, op.rhs[0]), np.linalg.solve(M, op2.rhs[0])]
    for k in range(2):
        assert rel(g[k], g_ref[k]) < 1e-8, k
    # element fields from the oracle's skeleton solution, on both sides
    g_or = np.stack(g_ref)
    u = solver.volume_solution(g_or, t=t, s=s)
    ts = [op.ts[0], op2.ts[0]]
    u_ref = oracle_fields(op, g_or, ts, fns)
    assert rel(u, u_ref) < 1e-10
    # and against the manufactured field itself (discretization error; resolved case only)
    if kappa < 20:
        X, Y = solver.node_coords()
        for k, th in enumerate(thetas):
            assert np.max(np.abs(u[k] - inputs.plane_wave(th, kappa, X, Y))) < 1e-5, k


@pytest.mark.parametrize("precision", [H.HPS_FP64, H.HPS_MIXED])
def test_volume_of_device_solution_and_scattered_field(solver, precision):
    """Scattered field s = -kappa^2 b e^{i kappa x}, t = 0 (the paper's experiment, section 5):
    u_scat + u_inc equals the total field of s = 0, t = I_i u_inc to the discretization error,
    and the device-resident path (device g, t, s, u) matches the oracle."""
    kappa, nx, N = 12.0, 4, 16
    bumps = [inputs.PAPER_BUMP]
    prob = inputs.Problem(nx=nx, N=N, kappa=kappa, eta=kappa, bumps=bumps, thetas=[0.0], L_exact=2)
    t_inc = H.setup(solver, prob, precision)
    solver.merge_levels(prob.L_exact)
    X, Y = solver.node_coords()
    fn = lambda X, Y: -kappa ** 2 * inputs.eval_b(bumps, X, Y) * np.exp(1j * kappa * X)  # noqa: E731
    s = torch.from_numpy(sources(solver, [fn])).cuda()
    t0 = torch.zeros((1, solver.n_bdry), dtype=torch.complex128, device="cuda")
    g_sc, info = solver.gmres_solve(t0, tol=1e-10, inner_iters=5, s=s)
    assert info["converged"] == 1 and info["max_rel_residual"] <= 1e-10
    u_sc = solver.volume_solution(g_sc, t=t0, s=s).cpu().numpy()
    g_tot, _ = solver.gmres_solve(t_inc, tol=1e-10, inner_iters=5)
    u_tot = solver.volume_solution(g_tot, t=t_inc)
    u_inc = inputs.plane_wave(0.0, kappa, X, Y)
    assert rel(u_sc[0] + u_inc, u_tot[0]) < 1e-6
    op = OracleProblem(inputs.Problem(nx=nx, N=N, kappa=kappa, eta=kappa, bumps=bumps, thetas=[0.0]), source=fn)
    u_ref = oracle_fields(op, g_sc.cpu().numpy(), [np.zeros(op.mesh.n_bdry, dtype=complex)], [fn])
    assert rel(u_sc, u_ref) < 1e-10


def test_64x64_N16_sources_sampled(solver):
    """Full-size manufactured problem: the FP64 residual of the source-driven solve and sampled
    element fields against the oracle's element solve."""
    prob = inputs.fp64_64x64(seed=1, nrhs=2)
    fns = [manufactured(prob.kappa, prob.bumps)(th) for th in prob.thetas]
    t = H.setup(solver, prob, H.HPS_MIXED)
    solver.merge_levels(prob.L_exact)
    s = torch.from_numpy(sources(solver, fns)).cuda()
    g, info = solver.gmres_solve(torch.from_numpy(t).cuda(), tol=1e-10, inner_iters=prob.inner_iters, s=s)
    assert info["converged"] == 2 and info["max_rel_residual"] <= 1e-10
    u = solver.volume_solution(g, t=torch.from_numpy(t).cuda(), s=s).cpu().numpy()
    gh = g.cpu().numpy()
    mesh = Mesh(64, 64, 16)
    w2 = interior_weights(16, mesh.h)
    rng = np.random.default_rng(3)
    for e in [0, 63, 2080, 4095] + [int(x) for x in rng.integers(0, 4096, 4)]:
        X, Y = mesh.node_xy(e)
        c = prob.kappa ** 2 * (1.0 - inputs.eval_b(prob.bumps, X, Y))
        for k in range(2):
            f_in = element_incoming(mesh, gh[k], t[k], e)
            ur = corner_values(16, leaf_solution(16, mesh.h, c, prob.eta, f_in, w2 * fns[k](X, Y)))
            assert rel(u[k, e], ur) < 1e-10, (e, k)
            assert np.max(np.abs(u[k, e] - inputs.plane_wave(prob.thetas[k], prob.kappa, X, Y))) < 1e-6
