"""Batching and serving: every result is the same alone and in the mix.

Batched runs build the leaves of a whole wave in one launch per GLL order and
overlap the problems' merges and solves on their own streams; the serving loop
batches requests for a cached tree into one multi-RHS solve.  Tolerances: the
same arithmetic per right-hand side (1e-12 relative for batches; 1e-8 for
served requests, whose FGMRES runs with other right-hand sides in lockstep so
split-K decisions may reorder sums), every solve at residual <= 1e-10, and
batched and served solutions within 1e-8 of the oracle's dense solve.
"""
import numpy as np
import pytest
import scipy.linalg as sla

torch = pytest.importorskip("torch")

from oracle.problem import OracleProblem
from oracle.skeleton import assemble_M
from paper_2511_00735_gb300 import batch as B
from paper_2511_00735_gb300 import hps as H
from paper_2511_00735_gb300 import inputs
from paper_2511_00735_gb300 import serve as S

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def mix():
    return [inputs.single_bump(4, 8, 10.0, 2, seed=31, L_exact=2),
            inputs.single_bump(8, 12, 30.0, 1, seed=32),
            inputs.single_bump(8, 8, 120.0, 3, seed=33),        # pivoted leaf route
            inputs.single_bump(16, 8, 40.0, 2, seed=34),
            inputs.single_bump(4, 16, 15.0, 1, seed=35, L_exact=3),
            inputs.single_bump(8, 16, 50.0, 2, seed=36)]


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("precision", [H.HPS_MIXED, H.HPS_FP64])
def test_batch_equals_alone(gpu, precision):
    probs = mix()
    br = B.BatchRunner(0, slots=4, precision=precision)
    res = br.run(probs)
    br.close()
    for p, (g, info) in zip(probs, res):
        g1, info1 = B.solve_alone(p, precision)
        assert max(info["rel_residual"]) <= 1e-10 and max(info1["rel_residual"]) <= 1e-10
        assert rel(g, g1) <= 1e-12, p.name


def test_batch_against_oracle(gpu):
    probs = mix()[:3]
    br = B.BatchRunner(0, slots=3, precision=H.HPS_MIXED)
    res = br.run(probs)
    br.close()
    for p, (g, _) in zip(probs, res):
        op = OracleProblem(p)
        M = assemble_M(op.mesh, op.Ts)
        for k in range(p.nrhs):
            assert rel(g[k], np.linalg.solve(M, op.rhs[k])) < 1e-8


def test_serve_same_alone_and_in_mix(gpu):
    rng = inputs.SplitMix64(77)
    bases = [inputs.single_bump(8, 8, 25.0, 1, seed=41), inputs.single_bump(8, 12, 30.0, 1, seed=42),
             inputs.single_bump(16, 8, 40.0, 1, seed=43), inputs.single_bump(4, 16, 15.0, 1, seed=44, L_exact=3)]
    reqs, t = [], 0.0
    for i in range(24):
        t += 0.002
        b = bases[rng.randint(0, 3)]
        th = [rng.uniform(0, 6.28) for _ in range(rng.randint(1, 4))]
        p = inputs.Problem(nx=b.nx, N=b.N, kappa=b.kappa, eta=b.eta, bumps=b.bumps, thetas=th, L_exact=b.L_exact,
                           inner_iters=b.inner_iters, name=b.name)
        reqs.append(S.Request(i, p, t))
    srv = S.Server(0, workers=3, precision=H.HPS_MIXED, hbm_cap=40e9)
    stats = S.run_stream(reqs, srv, timeout=300)
    srv.close()
    assert stats["requests"] == 24 and stats["max_rel_residual"] <= 1e-10
    assert stats["mean_batch"] > 1.0  # requests for a busy tree joined its next solve
    lus = {}
    for r in reqs:
        g1, info1 = B.solve_alone(r.prob, H.HPS_MIXED)
        assert max(info1["rel_residual"]) <= 1e-10
        assert rel(r.g, g1) <= 1e-8, r.rid
        # every served request against the oracle's dense solve of M g = RHS (one LU per tree)
        op = OracleProblem(r.prob)
        if r.prob.name not in lus:
            lus[r.prob.name] = sla.lu_factor(assemble_M(op.mesh, op.Ts))
        for k in range(r.prob.nrhs):
            assert rel(r.g[k], sla.lu_solve(lus[r.prob.name], op.rhs[k])) < 1e-8, (r.rid, k)


def test_admission_cap_evicts_idle_trees(gpu):
    bases = [inputs.single_bump(8, 8, 20.0 + 5 * i, 1, seed=50 + i) for i in range(5)]
    reqs = [S.Request(i, b, 0.001 * i) for i, b in enumerate(bases)]
    one = S.tree_bytes_estimate(8, 8, 1, H.HPS_MIXED)
    cap = 2.5 * one  # about two trees with their solve workspaces
    srv = S.Server(0, workers=1, precision=H.HPS_MIXED, hbm_cap=cap)
    stats = S.run_stream(reqs, srv, timeout=300)
    live, ev = len(srv.trees), srv.evictions
    srv.close()
    assert stats["requests"] == 5 and stats["max_rel_residual"] <= 1e-10
    assert stats["peak_device_bytes"] <= cap
    assert ev >= 1 and live + ev == 5   # five distinct trees could not all stay resident
