"""bench.py's algorithmic-bytes model of the V-cycle (the numerator of its HBM roofline) against
the merge tree the oracle builds (section 4.2: the nested-dissection merges and the coarse
subdomains), on small meshes with random leaf maps (the shapes do not depend on the values)."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402
from oracle.hps import MergeTree  # noqa: E402
from oracle.skeleton import Mesh  # noqa: E402


@pytest.mark.parametrize("nx,N,L_exact", [(4, 4, 2), (8, 4, 4), (8, 5, 3), (16, 3, 6)])
def test_vcycle_bytes_match_the_oracle_tree(nx, N, L_exact):
    mesh = Mesh(nx, nx, N)
    nb = 4 * (N - 1)
    rng = np.random.default_rng(nx * 100 + N)
    Ts = [0.1 * (rng.standard_normal((nb, nb)) + 1j * rng.standard_normal((nb, nb))) for _ in range(nx * nx)]
    tree = MergeTree(mesh, Ts, None, L_exact)
    ops = 0
    vec = 0
    for lev in range(1, L_exact + 1):
        for rec in tree.merges[lev]:
            n1, n2, m = rec.s1.n, rec.s2.n, rec.m
            outer = len(rec.E1) + len(rec.E2)
            # restriction U [outer x 2m] and prolongation Dm [2m x (n1 + n2)] of the pair
            ops += outer * 2 * m + 2 * m * (n1 + n2)
        rows_before = sum(s.n for s in tree.stages[lev - 1])
        vec += 2 * 2 * rows_before  # the stage vector read and written on the way up and down
    coarse = sum(int((s.inn >= 0).sum()) ** 2 for s in tree.stages[L_exact])
    vec += 2 * 2 * sum(s.n for s in tree.stages[0])  # the entry gather and the exit scatter
    nrhs, k = 7, 3
    got = bench.vcycle_bytes(nx, N, L_exact, nrhs, k)
    assert got["operator_bytes"] == 8 * (ops + k * coarse)
    assert got["vector_bytes"] == 8 * nrhs * vec
    assert got["bytes"] == got["operator_bytes"] + got["vector_bytes"]
