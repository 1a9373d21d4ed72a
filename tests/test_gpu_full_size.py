"""The 128x128-element, N = 16, kappa = 200 eight-bump workload (the benchmark's problem).

Sampled leaf maps against the oracle's dense leaf solve (section 3.1), the mixed-precision
solve's FP64 residual recomputed by the oracle's own skeleton operator and RHS (section 3.2)
from the library's leaf maps, and the mixed solution against the FP64 path's on the same
problem (section 4.3: the outer FP64 residual makes FGMRES an iterative refinement of the
FP32 tree, so both reach the same solution to about the tolerance times the conditioning).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.leaf import leaf_itI
from oracle.problem import plane_wave_data
from oracle.skeleton import Mesh, apply_M, assemble_rhs
from paper_2511_00735_gb300 import hps as H
from paper_2511_00735_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_128x128_N16_kappa200_mixed_against_oracle_and_fp64(gpu):
    prob = inputs.mixed_128x128(seed=2, nrhs=32)
    mesh = Mesh(prob.nx, prob.nx, prob.N)
    s = H.Solver(0)
    try:
        t = H.setup(s, prob, H.HPS_MIXED)
        # sampled leaves (corners, the bumps' centres, seeded others) against the oracle
        els = [0, prob.nx - 1, mesh.E - 1, mesh.E - prob.nx]
        for bp in prob.bumps:
            els.append(mesh.elem(min(int(bp.cx * prob.nx), prob.nx - 1), min(int(bp.cy * prob.nx), prob.nx - 1)))
        els += [int(e) for e in np.random.default_rng(5).integers(0, mesh.E, 8)]
        for e in els:
            X, Y = mesh.node_xy(e)
            c = prob.kappa ** 2 * (1.0 - inputs.eval_b(prob.bumps, X, Y))
            To = leaf_itI(prob.N, mesh.h, c, prob.eta)["T"]
            assert rel(s.leaf_T(e, 1)[0], To) < 1e-11, e
        s.merge_levels(prob.L_exact)
        g, info = s.gmres_solve(torch.from_numpy(t).cuda(), tol=1e-10, inner_iters=prob.inner_iters)
        g_mixed = g.cpu().numpy()
        assert info["converged"] == prob.nrhs and info["max_rel_residual"] <= 1e-10
        # the FP64 residual, by the oracle's operator on the library's (sample-checked) leaf maps
        Ts = list(s.leaf_T(0, mesh.E))
        rhs = np.stack([assemble_rhs(mesh, Ts, plane_wave_data(mesh, th, prob.kappa, prob.eta))
                        for th in prob.thetas], axis=1)
        r = rhs - apply_M(mesh, Ts, g_mixed.T)
        res = np.linalg.norm(r, axis=0) / np.linalg.norm(rhs, axis=0)
        assert np.max(np.abs(res - np.array(info["rel_residual"]))) <= 1e-14
        assert np.max(res) <= 1e-10 + 1e-14
        del Ts
        # the same problem on the FP64 path
        s.release_workspace()
        H.setup(s, prob, H.HPS_FP64)
        s.merge_levels(prob.L_exact)
        g64, info64 = s.gmres_solve(torch.from_numpy(t).cuda(), tol=1e-10, inner_iters=prob.inner_iters)
        assert info64["converged"] == prob.nrhs
        g64 = g64.cpu().numpy()
        err = max(rel(g_mixed[k], g64[k]) for k in range(prob.nrhs))
        print(f"128x128 N=16 kappa=200: mixed {info['outer_iterations']} its, FP64 {info64['outer_iterations']} its, "
              f"max rel l2 (mixed - FP64) = {err:.3e}")
        assert err < 1e-8
    finally:
        s.close()
