"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Every case is seeded and small enough for the oracle; tolerances follow from
FP64 rounding of the operations involved (relative l2 errors).  Index maps are
compared bit for bit.  The last test runs the 64x64, N = 16 workload and checks
sampled leaves against the oracle plus the explicit FP64 residual.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.hps import MergeTree
from oracle.leaf import leaf_itI
from oracle.problem import OracleProblem, coefficient
from oracle.skeleton import Mesh, apply_M, assemble_M
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


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def host(x):
    torch.cuda.synchronize()
    return x.cpu().numpy()


# ---------------------------------------------------------------- index maps
@pytest.mark.parametrize("nx,N", [(2, 3), (4, 6), (8, 4)])
def test_index_maps_bit_exact(solver, nx, N):
    solver.mesh(nx, N)
    sin, sout, bd = solver.index_maps()
    m = Mesh(nx, nx, N)
    q = N - 1
    e_in, e_out, e_bd = [], [], []
    for e in range(m.E):
        for s in range(4):
            for k in range(q):
                ui, uo, bi = m.unknown_in[e, s], m.unknown_out(e, s), m.bdry_in[e, s]
                e_in.append(ui + k if ui >= 0 else -1)
                e_out.append(uo + k if uo >= 0 else -1)
                e_bd.append(bi + k if bi >= 0 else -1)
    assert np.array_equal(sin, np.array(e_in)) and np.array_equal(sout, np.array(e_out))
    assert np.array_equal(bd, np.array(e_bd))
    X, Y = solver.node_coords()
    Xo, Yo = m.all_node_xy()
    np.testing.assert_allclose(X, Xo, atol=1e-15)
    np.testing.assert_allclose(Y, Yo, atol=1e-15)
    bx, by, bnx, bny = solver.boundary_points()
    ox, oy, onx, ony = m.boundary_points()
    np.testing.assert_allclose(np.stack([bx, by, bnx, bny]), np.stack([ox, oy, onx, ony]), atol=1e-15)


# ---------------------------------------------------------------- leaves
@pytest.mark.parametrize("nx,N,kappa", [(2, 4, 5.0), (4, 8, 10.0), (4, 16, 15.0), (8, 12, 30.0)])
def test_leaf_maps(solver, nx, N, kappa):
    prob = inputs.single_bump(nx, N, kappa, 1, seed=7)
    H.setup(solver, prob)
    Tg = solver.leaf_T(0, nx * nx)
    mesh = Mesh(nx, nx, N)
    c = coefficient(mesh, kappa, prob.bumps)
    for e in range(mesh.E):
        To = leaf_itI(N, mesh.h, c[e], kappa)["T"]
        assert rel(Tg[e], To) < 1e-11, e


@pytest.mark.parametrize("nx,N,kappa", [(2, 20, 5.0), (4, 24, 15.0), (2, 17, 8.0)])
def test_leaf_maps_high_order(solver, nx, N, kappa):
    """Orders above 16 (section 8(b) asks for N <= 24): the interior solver's leaf route
    (CG with fast diagonalisation, FP64 refinement) against the oracle's dense element solve."""
    prob = inputs.single_bump(nx, N, kappa, 1, seed=7)
    H.setup(solver, prob)
    Tg = solver.leaf_T(0, nx * nx)
    mesh = Mesh(nx, nx, N)
    c = coefficient(mesh, kappa, prob.bumps)
    for e in range(mesh.E):
        assert rel(Tg[e], leaf_itI(N, mesh.h, c[e], kappa)["T"]) < 1e-11, e


@pytest.mark.parametrize("precision", [H.HPS_FP64, H.HPS_MIXED])
def test_solve_order_24(solver, precision):
    """A 4x4, N=24 problem end to end (leaves by the interior solver, merges, FGMRES) against
    the oracle's dense skeleton solve; the elements away from the bump are past the
    positive-definite bound (kappa^2 (h/2)^2 = 6.25) and take the pivoted route."""
    prob = inputs.single_bump(4, 24, 20.0, 2, seed=13, L_exact=2)
    op = OracleProblem(prob)
    M = assemble_M(op.mesh, op.Ts)
    t = H.setup(solver, prob, precision)
    solver.merge_levels(prob.L_exact)
    g, info = solver.gmres_solve(t, tol=1e-10, inner_iters=5)
    assert info["converged"] == prob.nrhs and info["max_rel_residual"] <= 1e-10
    for k in range(prob.nrhs):
        assert rel(g[k], np.linalg.solve(M, op.rhs[k])) < 1e-8


@pytest.mark.parametrize("nx,N,kappa", [(2, 20, 100.0)])
def test_leaf_maps_robust_route_high_order(solver, nx, N, kappa):
    prob = inputs.Problem(nx=nx, N=N, kappa=kappa, eta=kappa, bumps=[inputs.PAPER_BUMP], thetas=[0.3])
    H.setup(solver, prob)
    op = OracleProblem(prob)
    Tg = solver.leaf_T(0, nx * nx)
    for e in range(nx * nx):
        assert rel(Tg[e], op.Ts[e]) < 1e-10, e


@pytest.mark.parametrize("nx,N,kappa", [(8, 8, 150.0), (8, 8, 36.0), (4, 12, 60.0)])
def test_leaf_maps_robust_route(solver, nx, N, kappa):
    # kappa^2 (1 - b) (h/2)^2 past the interior Dirichlet bound: the pivoted route (all
    # elements at kappa = 150; only those away from the bump at kappa = 36)
    prob = inputs.Problem(nx=nx, N=N, kappa=kappa, eta=kappa, bumps=[inputs.PAPER_BUMP], thetas=[0.1, 2.0],
                          L_exact=2)
    t = H.setup(solver, prob)
    op = OracleProblem(prob)
    Tg = solver.leaf_T(0, nx * nx)
    for e in range(nx * nx):
        assert rel(Tg[e], op.Ts[e]) < 1e-10, e
    M = assemble_M(op.mesh, op.Ts)
    solver.merge_levels(prob.L_exact)
    g, info = solver.gmres_solve(t, tol=1e-10, inner_iters=5, max_outer=40)
    for k in range(prob.nrhs):
        assert rel(g[k], np.linalg.solve(M, op.rhs[k])) < 1e-7
    assert info["max_rel_residual"] <= 1e-10


# ---------------------------------------------------------------- skeleton operators
@pytest.fixture(scope="module")
def cfg_small():
    prob = inputs.single_bump(4, 8, 12.0, 3, seed=11, L_exact=2)
    return prob, OracleProblem(prob)


def test_rhs_and_matvec(solver, cfg_small):
    prob, op = cfg_small
    t = H.setup(solver, prob)
    rhs = host(solver.rhs(dev(t)))
    for k in range(prob.nrhs):
        assert rel(rhs[k], op.rhs[k]) < 1e-12
    x = np.random.default_rng(0).standard_normal((3, op.mesh.n_skel)) * (1 - 0.7j)
    y = host(solver.matvec(dev(x)))
    yo = apply_M(op.mesh, op.Ts, x.T).T
    assert rel(y, yo) < 1e-12


def fp32_round(x):
    return (x.real.astype(np.float32) + 1j * x.imag.astype(np.float32)).astype(np.complex128)


@pytest.mark.parametrize("nx,N,kappa,nrhs", [(4, 8, 10.0, 3), (4, 12, 20.0, 16), (2, 16, 30.0, 20), (2, 24, 40.0, 32)])
def test_arnoldi_matvec_tensor_and_simt_vs_oracle(solver, nx, N, kappa, nrhs):
    """The mixed path's Arnoldi matvec (section 4.3, Pi M z with z in FP32) by exact splitting on
    the tensor cores and by double-float SIMT products, against the oracle's FP64 operator on the
    same FP32-rounded z.  Bound of the splitting: the 28 slice products with s + t <= 8 are exact,
    the dropped ones and the slices' truncation are below 2^-42 max|T_i.| max|z_.r| per k term
    (Ozaki et al. 2012), summed over the 8q real k; the SIMT path is double-float throughout."""
    prob = inputs.single_bump(nx, N, kappa, 1, seed=N)
    op = OracleProblem(prob)
    H.setup(solver, prob, H.HPS_MIXED)
    rng = np.random.default_rng(nrhs)
    # right-hand sides of very different scales and an all-zero one
    x = rng.standard_normal((nrhs, op.mesh.n_skel)) * (1 - 0.7j) * np.logspace(-20, 20, nrhs)[:, None]
    x[nrhs // 2] = 0.0
    xr = fp32_round(x)
    yo = apply_M(op.mesh, op.Ts, xr.T).T
    q = 4 * (N - 1)
    tmax = max(np.max(np.abs(T)) for T in op.Ts)
    try:
        for method, bound in ((H.MV_TENSOR, 2.0 ** -42 * 2 * q), (H.MV_SIMT, 2.0 ** -44 * 2 * q)):
            solver.set_arnoldi_matvec(method)
            y = host(solver.matvec_mixed(dev(x)))
            for k in range(nrhs):
                zmax = np.max(np.abs(xr[k]))
                err = np.max(np.abs(y[k] - yo[k]))
                assert err <= bound * tmax * zmax * 2 + 1e-300, (method, k, err, tmax * zmax)
                if zmax > 0:
                    assert rel(y[k], yo[k]) < 1e-12, (method, k)
                else:
                    assert np.all(y[k] == 0)
    finally:
        solver.set_arnoldi_matvec(H.MV_DEFAULT)


def test_mixed_solve_tensor_matvec_vs_simt(solver):
    """FGMRES on the mixed path with the tensor-core Arnoldi matvec and with the SIMT one: both
    reach the FP64 residual 1e-10, agree to the solve tolerance's conditioning and take the same
    number of iterations within one."""
    prob = inputs.single_bump(16, 16, 40.0, 24, seed=13, L_exact=6)
    t = H.setup(solver, prob, H.HPS_MIXED)
    solver.merge_levels(prob.L_exact)
    g, its = {}, {}
    try:
        for method in (H.MV_SIMT, H.MV_TENSOR):
            solver.set_arnoldi_matvec(method)
            g[method], info = solver.gmres_solve(t, tol=1e-10, inner_iters=prob.inner_iters, restart=20, max_outer=40)
            assert info["converged"] == prob.nrhs and info["max_rel_residual"] <= 1e-10, method
            its[method] = info["outer_iterations"]
    finally:
        solver.set_arnoldi_matvec(H.MV_DEFAULT)
    for k in range(prob.nrhs):
        assert rel(g[H.MV_TENSOR][k], g[H.MV_SIMT][k]) < 1e-8, k
    assert abs(its[H.MV_TENSOR] - its[H.MV_SIMT]) <= 1, its


# ---------------------------------------------------------------- merges
@pytest.mark.parametrize("nx,N,kappa", [(2, 6, 6.0), (4, 8, 10.0), (8, 4, 10.0)])
def test_stage_maps(solver, nx, N, kappa):
    prob = inputs.single_bump(nx, N, kappa, 1, seed=5)
    H.setup(solver, prob)
    op = OracleProblem(prob)
    L = op.mesh.L
    solver.merge_levels(L)
    tree = MergeTree(op.mesh, op.Ts, None, L)
    for k in range(L + 1):
        for sub in range(len(tree.stages[k])):
            Tg = solver.stage_T(k, sub)
            assert rel(Tg, tree.stages[k][sub].T) < 1e-10, (k, sub)


@pytest.mark.parametrize("L_exact", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("coarse", ["gmres", "exact"])
def test_precond_apply(solver, cfg_small, L_exact, coarse):
    prob, op = cfg_small
    H.setup(solver, prob)
    solver.merge_levels(L_exact, exact_coarse=(coarse == "exact"))
    tree = MergeTree(op.mesh, op.Ts, None, L_exact)
    r = np.random.default_rng(L_exact).standard_normal((2, op.mesh.n_skel)) * (0.3 + 1j)
    z = host(solver.precond_apply(dev(r), inner_iters=3))
    for k in range(2):
        zo = tree.mg(r[k], coarse, 3)
        assert rel(z[k], zo) < 1e-10, (L_exact, coarse, k)


# one bf16x3 sweep product: x = hi + lo to 2^-16 relative for each operand, and the dropped
# lo*lo term is below 2^-16: at most 3 * 2^-16 relative against the FP32 product
BF16X3_PRODUCT = 3 * 2.0 ** -16


@pytest.mark.parametrize("L_exact", [1, 2, 3])
@pytest.mark.parametrize("gamma", [2, 3])
@pytest.mark.parametrize("precision,sweep", [(H.HPS_FP64, H.SWEEP_DEFAULT), (H.HPS_MIXED, H.SWEEP_FP32),
                                             (H.HPS_MIXED, H.SWEEP_BF16X3)])
def test_precond_gamma_cycle(solver, cfg_small, L_exact, gamma, precision, sweep):
    """gamma coarse calls per level (section 4.3) against the oracle's gamma-cycle.  Tolerance:
    FP64 1e-10; FP32 tree 2e-5; bf16x3 sweeps add one product error per up- and down-sweep of
    every call of every level (level l runs gamma^l times), doubled."""
    prob, op = cfg_small
    H.setup(solver, prob, precision)
    solver.set_sweep_arith(sweep)
    try:
        solver.merge_levels(L_exact)
    finally:
        solver.set_sweep_arith(H.SWEEP_DEFAULT)
    tree = MergeTree(op.mesh, op.Ts, None, L_exact)
    r = np.random.default_rng(70 + L_exact).standard_normal((2, op.mesh.n_skel)) * (0.6 - 1j)
    solver.set_gamma(gamma)
    try:
        z = host(solver.precond_apply(dev(r), inner_iters=3))
    finally:
        solver.set_gamma(1)
    if precision == H.HPS_FP64:
        tol = 1e-10
    elif sweep == H.SWEEP_FP32:
        tol = 2e-5
    else:
        tol = 2e-5 + 2 * 2 * BF16X3_PRODUCT * sum(gamma ** lv for lv in range(L_exact))
    for k in range(2):
        zo = tree.mg(r[k], "gmres", 3, gamma)
        assert rel(z[k], zo) < tol, (L_exact, gamma, k)


def test_solve_gamma_cycle_mixed(solver):
    """FGMRES with the gamma = 2 cycle on the mixed path (the V-cycle graph with repeated coarse
    calls) reaches the dense solution and takes no more iterations than the V-cycle."""
    prob = inputs.single_bump(8, 12, 30.0, 2, seed=21, L_exact=4)
    op = OracleProblem(prob)
    M = assemble_M(op.mesh, op.Ts)
    t = H.setup(solver, prob, H.HPS_MIXED)
    solver.merge_levels(prob.L_exact)
    its = {}
    try:
        for gamma in (1, 2):
            solver.set_gamma(gamma)
            g, info = solver.gmres_solve(t, tol=1e-10, inner_iters=2)
            assert info["converged"] == prob.nrhs and info["max_rel_residual"] <= 1e-10
            for k in range(prob.nrhs):
                assert rel(g[k], np.linalg.solve(M, op.rhs[k])) < 1e-8
            its[gamma] = info["outer_iterations"]
    finally:
        solver.set_gamma(1)
    assert its[2] <= its[1], its


@pytest.mark.parametrize("sweep", [H.SWEEP_FP32, H.SWEEP_BF16X3])
@pytest.mark.parametrize("nrhs", [16, 32, 48])
def test_precond_mixed_tensor_core_sweeps(solver, nrhs, sweep):
    """FP32 tree on a 16x16, N=8 mesh: the upper sweep and coarse products (rows and k >= 64) run
    on the tensor cores (FP32 sweeps: 16, 32 or 64 column tiles; bf16x3 sweeps, on all six
    levels: 16 or 32 column tiles, side by side for 48); the V-cycle against the oracle's (section
    4.3).  Tolerance: 2e-5 for the FP32 tree; bf16x3 adds one product error on each up- and
    down-sweep, doubled for its growth through the coarse correction."""
    prob = inputs.single_bump(16, 8, 20.0, 1, seed=9, L_exact=6)
    op = OracleProblem(prob)
    H.setup(solver, prob, H.HPS_MIXED)
    solver.set_sweep_arith(sweep)
    try:
        solver.merge_levels(prob.L_exact)
    finally:
        solver.set_sweep_arith(H.SWEEP_DEFAULT)
    tree = MergeTree(op.mesh, op.Ts, None, prob.L_exact)
    r = np.random.default_rng(nrhs).standard_normal((nrhs, op.mesh.n_skel)) * (1 + 0.25j)
    z = host(solver.precond_apply(dev(r), inner_iters=4))
    tol = 2e-5 if sweep == H.SWEEP_FP32 else 2e-5 + 2 * 2 * prob.L_exact * BF16X3_PRODUCT
    for k in (0, nrhs // 2, nrhs - 1):
        assert rel(z[k], tree.mg(r[k], "gmres", 4)) < tol, k


def test_bf16x3_sweeps_against_fp32_sweeps_and_solve(solver):
    """32x32, N=16, kappa=60, 32 RHS, L_exact=8: the sweep products of every merge level run on the
    bf16x3 kernel (levels 1-3 with compact row tiles of 32-120 rows).  The V-cycle differs from
    the FP32-sweep V-cycle (itself pinned to the oracle above) by at most 2 products' error per
    level (up and down), doubled; both
    solves reach the FP64 residual 1e-10 and their solutions agree to the solve tolerance's
    conditioning; bf16x3 takes at most two more FGMRES iterations."""
    prob = inputs.single_bump(32, 16, 60.0, 32, seed=5, L_exact=8)
    t = H.setup(solver, prob, H.HPS_MIXED)
    r = np.random.default_rng(8).standard_normal((32, solver.n_skel)) * (0.3 + 1j)
    z, g, its = {}, {}, {}
    try:
        for sweep in (H.SWEEP_FP32, H.SWEEP_BF16X3):
            solver.set_sweep_arith(sweep)
            solver.merge_levels(prob.L_exact)
            z[sweep] = host(solver.precond_apply(dev(r), inner_iters=prob.inner_iters))
            g[sweep], info = solver.gmres_solve(t, tol=1e-10, inner_iters=prob.inner_iters)
            assert info["converged"] == 32 and info["max_rel_residual"] <= 1e-10, sweep
            its[sweep] = info["outer_iterations"]
    finally:
        solver.set_sweep_arith(H.SWEEP_DEFAULT)
    for k in (0, 13, 31):
        assert rel(z[H.SWEEP_BF16X3][k], z[H.SWEEP_FP32][k]) < 2 * 2 * prob.L_exact * BF16X3_PRODUCT, k
        assert rel(g[H.SWEEP_BF16X3][k], g[H.SWEEP_FP32][k]) < 1e-8, k
    assert its[H.SWEEP_BF16X3] <= its[H.SWEEP_FP32] + 2, its


def test_precond_exact_is_inverse(solver, cfg_small):
    prob, op = cfg_small
    H.setup(solver, prob)
    solver.merge_levels(op.mesh.L)
    r = np.random.default_rng(3).standard_normal((1, op.mesh.n_skel)) + 0j
    z = host(solver.precond_apply(dev(r)))
    assert rel(z[0], np.linalg.solve(assemble_M(op.mesh, op.Ts), r[0])) < 1e-11


# ---------------------------------------------------------------- solves
def test_solve_4x4_fp64(solver):
    prob = inputs.small_4x4(0)
    op = OracleProblem(prob)
    g_ref = np.linalg.solve(assemble_M(op.mesh, op.Ts), op.rhs[0])
    t = H.setup(solver, prob)
    solver.merge_levels(prob.L_exact)
    g, info = solver.gmres_solve(t, tol=1e-10, inner_iters=prob.inner_iters)
    assert info["max_rel_residual"] <= 1e-10
    assert rel(g[0], g_ref) < 1e-9
    _, oinfo = op.solve_fgmres(L_exact=prob.L_exact, inner_iters=prob.inner_iters, tol=1e-10)
    assert abs(info["outer_iterations"] - oinfo[0]["iterations"]) <= 1
    # direct HPS: all merges but the last, exact coarse -> one iteration
    solver.merge_levels(op.mesh.L - 1, exact_coarse=True)
    g2, info2 = solver.gmres_solve(t, tol=1e-10, inner_iters=0)
    assert info2["outer_iterations"] == 1 and rel(g2[0], g_ref) < 1e-10


def test_solve_unpreconditioned_and_multi_rhs(solver, cfg_small):
    prob, op = cfg_small
    t = H.setup(solver, prob)
    g, info = solver.gmres_solve(t, tol=1e-10, inner_iters=-1, restart=30, max_outer=40)
    M = assemble_M(op.mesh, op.Ts)
    for k in range(prob.nrhs):
        assert rel(g[k], np.linalg.solve(M, op.rhs[k])) < 1e-8
    assert info["max_rel_residual"] <= 1e-10


@pytest.mark.parametrize("precision", [H.HPS_FP64, H.HPS_MIXED])
def test_solve_8x8_device_buffers(solver, precision):
    prob = inputs.single_bump(8, 12, 30.0, 4, seed=21, L_exact=4)
    op = OracleProblem(prob)
    M = assemble_M(op.mesh, op.Ts)
    t = H.setup(solver, prob, precision)
    solver.merge_levels(prob.L_exact)
    g, info = solver.gmres_solve(dev(t), tol=1e-10, inner_iters=5)
    g = host(g)
    assert info["max_rel_residual"] <= 1e-10
    for k in range(prob.nrhs):
        gr = np.linalg.solve(M, op.rhs[k])
        assert rel(g[k], gr) < 1e-8
        assert np.linalg.norm(op.rhs[k] - M @ g[k]) / np.linalg.norm(op.rhs[k]) < 1e-9


@pytest.mark.parametrize("inner", [5, -1])
def test_solve_outer_df64_vs_fp64(solver, inner):
    """Mixed path, outer FGMRES in double-float arithmetic against the same solve in FP64
    (section 4.3): both reach the tolerance on the FP64 residual, both match the oracle's
    dense solve, and their iteration counts differ by at most a few."""
    prob = inputs.single_bump(8, 12, 30.0, 4, seed=21, L_exact=4)
    op = OracleProblem(prob)
    M = assemble_M(op.mesh, op.Ts)
    t = H.setup(solver, prob, H.HPS_MIXED)
    solver.merge_levels(prob.L_exact)
    its = {}
    try:
        for mode in (H.OUTER_FP64, H.OUTER_DF64):
            solver.set_outer_arith(mode)
            g, info = solver.gmres_solve(t, tol=1e-10, inner_iters=inner, restart=60, max_outer=20)
            assert info["converged"] == prob.nrhs and info["max_rel_residual"] <= 1e-10
            for k in range(prob.nrhs):
                gr = np.linalg.solve(M, op.rhs[k])
                assert rel(g[k], gr) < 1e-8
                assert np.linalg.norm(op.rhs[k] - M @ g[k]) / np.linalg.norm(op.rhs[k]) < 1e-9
            its[mode] = info["outer_iterations"]
    finally:
        solver.set_outer_arith(H.OUTER_DEFAULT)
    assert abs(its[H.OUTER_FP64] - its[H.OUTER_DF64]) <= max(2, its[H.OUTER_FP64] // 20), its


def test_outer_df64_needs_mixed_leaves(solver):
    prob = inputs.small_4x4(0)
    t = H.setup(solver, prob, H.HPS_FP64)
    solver.merge_levels(prob.L_exact)
    with pytest.raises(H.HPSError):
        solver.set_outer_arith(7)
    solver.set_outer_arith(H.OUTER_DF64)
    try:
        with pytest.raises(H.HPSError):
            solver.gmres_solve(t, tol=1e-10, inner_iters=prob.inner_iters)
    finally:
        solver.set_outer_arith(H.OUTER_DEFAULT)
    g, info = solver.gmres_solve(t, tol=1e-10, inner_iters=prob.inner_iters)
    assert info["max_rel_residual"] <= 1e-10


def test_merges_mixed_tensor_cores(solver):
    """Mixed-precision merge tree (FP32; the top merge of a 16x16, N=8 mesh runs its GEMMs on
    the tensor cores, 3xTF32) against the FP64 tree and the oracle (section 4.1)."""
    prob = inputs.single_bump(16, 8, 20.0, 1, seed=9)
    L = 8
    H.setup(solver, prob, H.HPS_FP64)
    solver.merge_levels(L)
    top = [(k, sub) for k in (L - 1, L) for sub in range(2 ** (L - k))]
    ref = {ks: solver.stage_T(*ks) for ks in top}
    H.setup(solver, prob, H.HPS_MIXED)
    solver.merge_levels(L)
    for ks in top:
        assert rel(solver.stage_T(*ks), ref[ks]) < 2e-5, ks
    op = OracleProblem(prob)
    tree = MergeTree(op.mesh, op.Ts, None, L)
    assert rel(solver.stage_T(L, 0), tree.stages[L][0].T) < 2e-5


def test_bad_arguments(solver):
    with pytest.raises(H.HPSError):
        solver.mesh(6, 8)
    with pytest.raises(H.HPSError):
        solver.mesh(4, 25)
    solver.mesh(4, 8)
    with pytest.raises(H.HPSError):
        solver.build_leaves()          # no coefficient yet
    with pytest.raises(H.HPSError):
        solver.merge_levels(1)


# ---------------------------------------------------------------- full size
def test_64x64_N16_sampled(solver):
    prob = inputs.fp64_64x64(seed=1, nrhs=4)
    t = H.setup(solver, prob, H.HPS_FP64)
    mesh = Mesh(64, 64, 16)
    c = coefficient(mesh, prob.kappa, prob.bumps)
    rng = np.random.default_rng(0)
    for e in [0, 63, 4095, 2080] + list(rng.integers(0, 4096, 6)):
        To = leaf_itI(16, mesh.h, c[e], prob.kappa)["T"]
        assert rel(solver.leaf_T(int(e), 1)[0], To) < 1e-11, e
    solver.merge_levels(prob.L_exact)
    g, info = solver.gmres_solve(dev(t), tol=1e-10, inner_iters=prob.inner_iters)
    assert info["converged"] == prob.nrhs and info["max_rel_residual"] <= 1e-10
    rhs = solver.rhs(dev(t))
    r = host(rhs) - host(solver.matvec(g))
    res = np.linalg.norm(r, axis=1) / np.linalg.norm(host(rhs), axis=1)
    # the reported residual is the FP64 residual of the returned solution (summation order aside)
    assert np.max(np.abs(res - np.array(info["rel_residual"]))) <= 1e-15
    assert np.max(res) <= 1e-10 + 1e-15


def test_64x64_N16_mixed_residual_in_fp64(solver):
    """Mixed path at 64x64 (FP32 tree and sweeps, double-float Arnoldi steps): the residual the
    solve reports is the FP64 residual of the solution it returns, recomputed here through the
    FP64 RHS and matvec entry points, and it meets the 1e-10 tolerance with no slack (section
    4.3: FGMRES as iterative refinement)."""
    prob = inputs.fp64_64x64(seed=1, nrhs=4)
    t = H.setup(solver, prob, H.HPS_MIXED)
    solver.merge_levels(prob.L_exact)
    g, info = solver.gmres_solve(dev(t), tol=1e-10, inner_iters=prob.inner_iters)
    assert info["converged"] == prob.nrhs and info["max_rel_residual"] <= 1e-10
    rhs = solver.rhs(dev(t))
    r = host(rhs) - host(solver.matvec(g))
    res = np.linalg.norm(r, axis=1) / np.linalg.norm(host(rhs), axis=1)
    # the reported residual is the FP64 residual of the returned solution (summation order aside)
    assert np.max(np.abs(res - np.array(info["rel_residual"]))) <= 1e-15
    assert np.max(res) <= 1e-10 + 1e-15


def _level_shapes(nx, q, L_exact):
    """(pairs, n, m, p) of merge levels 1..L_exact of an nx x nx mesh: a child's boundary length n,
    its interface length m (the merged side, alternately vertical and horizontal), p = n - m."""
    a = b = 1
    out = []
    for lev in range(1, L_exact + 1):
        n = 2 * (a + b) * q
        m = (b if lev % 2 == 1 else a) * q
        out.append(((nx * nx) >> lev, n, m, n - m))
        if lev % 2 == 1:
            a *= 2
        else:
            b *= 2
    return out


@pytest.mark.parametrize("cand", range(6))
@pytest.mark.parametrize("sweep,nrhs", [(H.SWEEP_BF16X3, 32), (H.SWEEP_BF16X3, 48), (H.SWEEP_FP32, 32)])
def test_autotune_every_candidate_vs_oracle(solver, cand, sweep, nrhs):
    """Every launch configuration the tile autotuner can pick (forced with TUNE_FORCE + i: column
    tiles of half width, one CTA per SM, no or twice the k split) for the merge GEMMs and the sweep
    products of the 16x16, N=8 tree: the V-cycle against the oracle's to the tolerance of the
    default configuration (the candidates differ only in tiling and in the k summation order)."""
    prob = inputs.single_bump(16, 8, 20.0, 1, seed=9, L_exact=6)
    op = OracleProblem(prob)
    H.setup(solver, prob, H.HPS_MIXED)
    solver.set_sweep_arith(sweep)
    solver.set_autotune(H.TUNE_FORCE + cand)
    try:
        solver.merge_levels(prob.L_exact)
        r = np.random.default_rng(100 + cand).standard_normal((nrhs, op.mesh.n_skel)) * (1 - 0.5j)
        z = host(solver.precond_apply(dev(r), inner_iters=4))
    finally:
        solver.set_autotune(H.TUNE_OFF)
        solver.set_sweep_arith(H.SWEEP_DEFAULT)
    tree = MergeTree(op.mesh, op.Ts, None, prob.L_exact)
    tol = 2e-5 if sweep == H.SWEEP_FP32 else 2e-5 + 2 * 2 * prob.L_exact * BF16X3_PRODUCT
    for k in (0, nrhs - 1):
        assert rel(z[k], tree.mg(r[k], "gmres", 4)) < tol, (cand, k)


def test_autotune_on_tunes_once_and_solves(solver):
    """TUNE_ON on the 32x32, N=16, kappa=60 tree with 32 RHS: the merges and the first V-cycle tune
    their GEMM shapes (the table gains tc and tcb entries), a second tree build and V-cycle add none,
    the tuned V-cycle agrees with the untuned one within twice the FP32/bf16x3 tree's error bound,
    and FGMRES reaches the FP64 residual 1e-10 within one iteration of the untuned solve."""
    prob = inputs.single_bump(32, 16, 60.0, 32, seed=5, L_exact=8)
    t = H.setup(solver, prob, H.HPS_MIXED)
    r = np.random.default_rng(81).standard_normal((32, solver.n_skel)) * (1 + 0.2j)
    H.autotune_clear()
    z, its = {}, {}
    try:
        for mode in (H.TUNE_OFF, H.TUNE_ON):
            solver.set_autotune(mode)
            solver.merge_levels(prob.L_exact)
            z[mode] = host(solver.precond_apply(dev(r), inner_iters=prob.inner_iters))
            g, info = solver.gmres_solve(t, tol=1e-10, inner_iters=prob.inner_iters, restart=20)
            assert info["converged"] == 32 and info["max_rel_residual"] <= 1e-10, mode
            its[mode] = info["outer_iterations"]
        table = H.autotune_table()
        n_shapes = len(table.splitlines())
        assert any(line.startswith("tcb ") for line in table.splitlines()), table
        assert any(line.startswith("tc ") for line in table.splitlines()), table
        solver.merge_levels(prob.L_exact)
        solver.precond_apply(dev(r), inner_iters=prob.inner_iters)
        assert len(H.autotune_table().splitlines()) == n_shapes
    finally:
        solver.set_autotune(H.TUNE_OFF)
    tol = 2 * (2e-5 + 2 * 2 * prob.L_exact * BF16X3_PRODUCT)
    for k in (0, 17, 31):
        assert rel(z[H.TUNE_ON][k], z[H.TUNE_OFF][k]) < tol, k
    assert abs(its[H.TUNE_ON] - its[H.TUNE_OFF]) <= 1, its


def test_profile_kernels_sweep_and_merge_classes(solver):
    """hps_profile_kernels on the 16x16, N=8 mixed tree (bf16x3 sweeps on all six levels) with 24
    RHS: two direct V-cycles bracket 2 x 2 x 6 sweep launches whose algorithmic bytes are the
    operators U [2p x 2m] and Dm [2m x 2n] of every pair at 8 B per complex entry plus B, C0 (up-sweep
    only) and C at 8 B per entry each; the tree build brackets its merge GEMMs with positive flops;
    launches captured into the solve's V-cycle graph are not bracketed."""
    prob = inputs.single_bump(16, 8, 20.0, 1, seed=9, L_exact=6)
    t = H.setup(solver, prob, H.HPS_MIXED)
    nrhs = 24
    r = np.random.default_rng(3).standard_normal((nrhs, solver.n_skel)) + 0j
    solver.profile_kernels(True)
    try:
        solver.merge_levels(prob.L_exact)
        for _ in range(2):
            solver.precond_apply(dev(r), inner_iters=3)
        d = solver.profile_kernels_read()
    finally:
        solver.profile_kernels(False)
    want = 0.0
    for npairs, n, m, p in _level_shapes(16, prob.N - 1, prob.L_exact):
        want += 8.0 * npairs * (2 * p * 2 * m + 2 * m * nrhs + 2 * 2 * p * nrhs)  # up: C0 and C of 2p rows
        want += 8.0 * npairs * (2 * m * 2 * n + 2 * n * nrhs + 2 * m * nrhs)      # down
    ms, launches, nbytes, flops = d["sweep"]
    assert launches == 2 * 2 * prob.L_exact and ms > 0
    assert nbytes == pytest.approx(2 * want, rel=1e-12)
    ms_m, launches_m, _, flops_m = d["merge_gemm"]
    assert launches_m > 0 and flops_m > 0 and ms_m > 0
    # a solve replays the V-cycle as a graph: none of its sweep launches is bracketed
    solver.profile_kernels(True)
    try:
        solver.gmres_solve(t, tol=1e-10, inner_iters=3, restart=20)
        d2 = solver.profile_kernels_read()
    finally:
        solver.profile_kernels(False)
    assert d2["sweep"][1] == 0
