"""The allocation-free leaf entry point matches hps_build_leaves.

hps_leaf_maps_noalloc serves callers that cannot allocate device memory while
they run (their device memory belongs to their own pool, or they must not
trigger the implicit synchronisation of cudaMalloc/cudaFree).  It keeps its
workspace in a static device array shared by every call, so two calls in a
row must give the same maps as the allocating path.  This file runs last
(pytest collects files alphabetically) so that a failure here does not hide
the other GPU tests.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2511_00735_gb300 import hps as H
from paper_2511_00735_gb300 import inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("nx,N,kappa", [(4, 8, 10.0), (8, 16, 30.0)])
def test_noalloc_leaf_maps_match_allocating_path(nx, N, kappa):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    prob = inputs.single_bump(nx, N, kappa, 1, seed=9)
    s = H.Solver(0)
    H.setup(s, prob)
    T_ref = s.leaf_T(0, nx * nx)
    X, Y = s.node_coords()
    s.close()
    c = torch.from_numpy(kappa ** 2 * (1.0 - inputs.eval_b(prob.bumps, X, Y))).cuda().contiguous()
    lib = H.load_library()
    stream = torch.cuda.current_stream().cuda_stream
    nb = 4 * (N - 1)
    for _ in range(2):  # two calls in a row share the static workspace
        T = torch.full((nx * nx, nb, nb), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
        st = lib.hps_leaf_maps_noalloc(0, ctypes.c_void_p(stream), N, 1.0 / nx, kappa, ctypes.c_void_p(c.data_ptr()),
                                       nx * nx, ctypes.c_void_p(T.data_ptr()))
        assert st == 0
        torch.cuda.synchronize()
        Tn = T.cpu().numpy()
        for e in range(nx * nx):
            assert rel(Tn[e], T_ref[e]) < 1e-11, e


def test_noalloc_rejects_orders_beyond_the_workspace():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = H.load_library()
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    assert lib.hps_leaf_maps_noalloc(0, None, 17, 0.25, 10.0, ctypes.c_void_p(dummy.data_ptr()), 1,
                                     ctypes.c_void_p(dummy.data_ptr())) == -1
