"""Pins of the oracle's merges, nested dissection and multigrid preconditioner (section 4)."""
import json
import os

import numpy as np
import pytest

from oracle.hps import MergeTree, mg_dense, schur_levels, unknown_levels
from oracle.problem import OracleProblem
from oracle.skeleton import Mesh, assemble_M
from paper_2511_00735_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def small():
    p = inputs.Problem(nx=4, N=6, kappa=10.0, eta=10.0, bumps=[inputs.PAPER_BUMP], thetas=[0.4])
    op = OracleProblem(p)
    M = assemble_M(op.mesh, op.Ts)
    return op, M, unknown_levels(op.mesh)


def test_merge_equals_dense_schur(small):
    # eq. globalfacesystem (local merges) == block elimination of the assembled M
    op, M, lv = small
    ms = schur_levels(M, lv, op.mesh.L - 1)
    for L_exact in range(1, op.mesh.L):
        tree = MergeTree(op.mesh, op.Ts, None, L_exact)
        cidx = tree.coarse_index()
        Mc = tree.coarse_dense(cidx)
        S, _ = ms[L_exact]
        assert S.shape == Mc.shape
        assert np.linalg.norm(Mc - S) / np.linalg.norm(S) < 1e-13


def test_merge_2x2_mesh():
    p = inputs.Problem(nx=2, N=8, kappa=12.0, eta=12.0, bumps=[inputs.PAPER_BUMP], thetas=[1.0])
    op = OracleProblem(p)
    M = assemble_M(op.mesh, op.Ts)
    lv = unknown_levels(op.mesh)
    S, _ = schur_levels(M, lv, 1)[1]
    tree = MergeTree(op.mesh, op.Ts, None, 1)
    assert np.linalg.norm(tree.coarse_dense(tree.coarse_index()) - S) / np.linalg.norm(S) < 1e-13


def _face_of(mesh, ea, eb):
    # paper labels: elements 1-based, x fastest
    a, b = ea - 1, eb - 1
    for f, (e1, _, e2, _) in enumerate(mesh.faces):
        if {e1, e2} == {a, b}:
            return f
    raise KeyError((ea, eb))


def test_fig1_sparsity_patterns(small):
    op, M, lv = small
    mesh, q = op.mesh, op.mesh.q
    fx = json.load(open(os.path.join(HERE, "golden", "fig1_sparsity.json")))
    ms = schur_levels(M, lv, 3)
    for g in ("1", "2", "3", "4"):
        Ml, lvl = ms[int(g) - 1]
        # global unknown ids kept in M_l, in increasing order
        keep = np.where(lv >= int(g))[0]
        pos = {u: i for i, u in enumerate(keep)}
        grid = fx["grids"][g]
        label_face = {lab: _face_of(mesh, ea, eb) for lab, ea, eb in grid["faces"]}
        # every face of this grid is a face remaining at level g
        assert sorted(label_face.values()) == sorted(
            {f for f in range(mesh.nfaces) if mesh.face_level(f) >= int(g)})

        def rows_of(labels):
            out = []
            for lab in labels:
                f = label_face[lab]
                out += [pos[u] for u in range(2 * f * q, (2 * f + 2) * q)]
            return out

        units = ([[lab] for lab in range(1, len(grid["faces"]) + 1)] if grid["granularity"] == "face"
                 else grid["groups"])
        for blk in "ABCD":
            spec = grid[blk]
            want = {tuple(c) for c in spec["cells"]}
            if grid["granularity"] == "face":
                R = [[lab] for lab in spec["rows"]]
                C = [[lab] for lab in spec["cols"]]
            else:
                R = [units[i - 1] for i in spec["rows"]]
                C = [units[i - 1] for i in spec["cols"]]
            got = set()
            for i, rl in enumerate(R):
                for j, cl in enumerate(C):
                    sub = Ml[np.ix_(rows_of(rl), rows_of(cl))]
                    if np.abs(sub).max() > 1e-12 * np.abs(Ml).max():
                        got.add((i + 1, j + 1))
            assert got == want, (g, blk, sorted(got ^ want))


@pytest.mark.parametrize("L_exact", [0, 1, 2, 3])
def test_mg_structured_equals_literal_formula(small, L_exact):
    op, M, lv = small
    tree = MergeTree(op.mesh, op.Ts, None, L_exact)
    r = np.random.default_rng(L_exact).standard_normal(op.mesh.n_skel) * (1 - 0.5j)
    for coarse in ("gmres", "exact"):
        zd = mg_dense(M, lv, 1, L_exact, r, coarse, 4)
        zs = tree.mg(r, coarse, 4)
        assert np.linalg.norm(zs - zd) / np.linalg.norm(zd) < 1e-12


@pytest.mark.parametrize("L_exact", [0, 1, 2, 3])
def test_exact_coarse_is_inverse(small, L_exact):
    # block-inverse identity: with an exact coarse solve MG(M) = M^{-1}
    op, M, lv = small
    tree = MergeTree(op.mesh, op.Ts, None, L_exact)
    r = np.random.default_rng(10 + L_exact).standard_normal(op.mesh.n_skel) + 0j
    z = tree.mg(r, "exact")
    zt = np.linalg.solve(M, r)
    assert np.linalg.norm(z - zt) / np.linalg.norm(zt) < 1e-12


def test_restriction_identity(small):
    # (I - M F) r has an exactly zero A-block at every level
    op, M, lv = small
    r = np.random.default_rng(5).standard_normal(op.mesh.n_skel) + 1j
    for lev in (1, 2):
        Ml, lvl = schur_levels(M, lv, lev - 1)[lev - 1]
        rl = r[: len(lvl)]
        xs = np.where(lvl == lev)[0]
        Fr = np.zeros_like(rl)
        Fr[xs] = np.linalg.solve(Ml[np.ix_(xs, xs)], rl[xs])
        res = rl - Ml @ Fr
        assert np.abs(res[xs]).max() < 1e-13 * np.abs(rl).max()


def test_transposed_child_map_fails_dense_schur(small, monkeypatch):
    # planted mistake: a merge that reads its children's maps transposed no longer equals the
    # block elimination of the assembled M (the pin above would catch it)
    import oracle.hps as hps_mod

    op, M, lv = small
    orig = hps_mod.merge_pair

    def transposed(mesh, s1, s2, direction, keep_blocks=True):
        t1, t2 = s1.T, s2.T
        s1.T, s2.T = t1.T.copy(), t2.T.copy()
        try:
            return orig(mesh, s1, s2, direction, keep_blocks)
        finally:
            s1.T, s2.T = t1, t2

    monkeypatch.setattr(hps_mod, "merge_pair", transposed)
    S, _ = schur_levels(M, lv, 1)[1]
    tree = hps_mod.MergeTree(op.mesh, op.Ts, None, 1)
    assert np.linalg.norm(tree.coarse_dense(tree.coarse_index()) - S) / np.linalg.norm(S) > 1e-3


def test_transposed_interface_solve_fails_block_inverse(small, monkeypatch):
    # planted mistake: the sweeps solving with A^T instead of A break MG(M) = M^{-1} for an
    # exact coarse solve (the block-inverse pin above would catch it)
    import scipy.linalg as sla

    import oracle.hps as hps_mod

    op, M, lv = small
    monkeypatch.setattr(hps_mod.MergeRecord, "solveA", lambda self, v: sla.lu_solve(self.lu, v, trans=1))
    tree = hps_mod.MergeTree(op.mesh, op.Ts, None, 2)
    r = np.random.default_rng(12).standard_normal(op.mesh.n_skel) + 0j
    z = tree.mg(r, "exact")
    zt = np.linalg.solve(M, r)
    assert np.linalg.norm(z - zt) / np.linalg.norm(zt) > 1e-3


# ---------------------------------------------------------------- gamma-cycle (section 4.3)
@pytest.mark.parametrize("L_exact", [1, 2, 3])
@pytest.mark.parametrize("gamma", [2, 3])
def test_gamma_cycle_structured_equals_literal_formula(small, L_exact, gamma):
    # the per-pair recursion against the literal recursion on the assembled M: two independent
    # statements of e_k = e_{k-1} + MG(S)(r_c - S e_{k-1}) (GMRES coarse solve: nonlinear in r)
    op, M, lv = small
    tree = MergeTree(op.mesh, op.Ts, None, L_exact)
    r = np.random.default_rng(20 + L_exact).standard_normal(op.mesh.n_skel) * (0.4 - 1j)
    zd = mg_dense(M, lv, 1, L_exact, r, "gmres", 3, gamma)
    zs = tree.mg(r, "gmres", 3, gamma)
    assert np.linalg.norm(zs - zd) / np.linalg.norm(zd) < 1e-12


@pytest.mark.parametrize("L_exact", [0, 1, 2])
def test_gamma_one_is_the_v_cycle(small, L_exact):
    op, M, lv = small
    tree = MergeTree(op.mesh, op.Ts, None, L_exact)
    r = np.random.default_rng(30 + L_exact).standard_normal(op.mesh.n_skel) + 0.3j
    assert np.linalg.norm(tree.mg_gamma(r, "gmres", 4, 1) - tree.mg(r, "gmres", 4)) <= 1e-13 * np.linalg.norm(r)


@pytest.mark.parametrize("gamma", [2, 3])
def test_gamma_cycle_exact_coarse_is_inverse(small, gamma):
    # with an exact coarse solve every coarse call is exact, the later calls correct nothing,
    # and the gamma-cycle is M^{-1} like the V-cycle (block-inverse identity)
    op, M, lv = small
    tree = MergeTree(op.mesh, op.Ts, None, 2)
    r = np.random.default_rng(40 + gamma).standard_normal(op.mesh.n_skel) + 0j
    z = tree.mg(r, "exact", 0, gamma)
    zt = np.linalg.solve(M, r)
    assert np.linalg.norm(z - zt) / np.linalg.norm(zt) < 1e-12


def test_gamma_cycle_contracts_toward_the_inverse(small):
    # more coarse calls per level move MG(M) r closer to M^{-1} r for a fixed coarse solver
    # (each call is one step of a convergent iteration on the coarse-level system)
    op, M, lv = small
    tree = MergeTree(op.mesh, op.Ts, None, 2)
    r = np.random.default_rng(50).standard_normal(op.mesh.n_skel) * (1 + 0.5j)
    zt = np.linalg.solve(M, r)
    errs = [np.linalg.norm(tree.mg(r, "gmres", 2, g) - zt) / np.linalg.norm(zt) for g in (1, 2, 4)]
    assert errs[0] > errs[1] > errs[2], errs


def test_gamma_cycle_without_residual_update_fails(small, monkeypatch):
    # planted mistake: coarse calls that all take the restricted residual r_c (no "- S e")
    # add up to gamma MG(S) r_c; the structured-vs-literal pin above catches it
    import oracle.hps as hps_mod

    op, M, lv = small
    tree = hps_mod.MergeTree(op.mesh, op.Ts, None, 2)
    monkeypatch.setattr(hps_mod.MergeTree, "stage_apply", lambda self, k, g: np.zeros_like(g))
    r = np.random.default_rng(60).standard_normal(op.mesh.n_skel) + 0j
    zd = mg_dense(M, lv, 1, 2, r, "gmres", 3, 2)
    zs = tree.mg(r, "gmres", 3, 2)
    assert np.linalg.norm(zs - zd) / np.linalg.norm(zd) > 1e-3
