"""The allocation-free leaf entry point matches hps_build_leaves.

hps_leaf_maps_noalloc serves callers that cannot allocate device memory while
they run (their device memory belongs to their own pool, or they must not
trigger the implicit synchronisation of cudaMalloc/cudaFree).  It keeps its
workspace in a static device array shared by every call, so two calls in a
row must give the same maps as the allocating path, and a call after the first
must leave the device's free memory unchanged.  This file runs last (pytest
collects files alphabetically) so that a failure here does not hide the other
GPU tests.
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


def call(lib, N, h, eta, c, E, T):
    stream = torch.cuda.current_stream().cuda_stream
    return lib.hps_leaf_maps_noalloc(0, ctypes.c_void_p(stream), N, h, eta, ctypes.c_void_p(c.data_ptr()), E,
                                     ctypes.c_void_p(T.data_ptr()))


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
    nb = 4 * (N - 1)
    outs = [torch.full((nx * nx, nb, nb), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
            for _ in range(2)]
    torch.cuda.synchronize()
    for k, T in enumerate(outs):  # two calls in a row share the static workspace
        free0 = torch.cuda.mem_get_info(0)[0]
        assert call(lib, N, 1.0 / nx, kappa, c, nx * nx, T) == 0
        torch.cuda.synchronize()
        if k == 1:  # after the first call (module load, symbol lookup) no call changes free device memory
            assert torch.cuda.mem_get_info(0)[0] == free0
        Tn = T.cpu().numpy()
        for e in range(nx * nx):
            assert rel(Tn[e], T_ref[e]) < 1e-11, e


def test_noalloc_reports_an_indefinite_interior_operator():
    """kappa^2 (h/2)^2 = 25 is far above the smallest interior eigenvalue of the reference
    element (about 4.9): the real L D L^T meets a negative pivot, and this entry, which has
    no pivoted route, reports HPS_ENUMERIC (its maps are then undefined)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nx, N, kappa = 4, 8, 40.0
    lib = H.load_library()
    c = torch.full((nx * nx, (N + 1) ** 2), kappa ** 2, dtype=torch.float64, device="cuda")
    T = torch.zeros((nx * nx, 4 * (N - 1), 4 * (N - 1)), dtype=torch.complex128, device="cuda")
    assert call(lib, N, 1.0 / nx, kappa, c, nx * nx, T) == H.HPS_ENUMERIC
    torch.cuda.synchronize()
    assert torch.cuda.current_device() == 0


def test_noalloc_rejects_orders_beyond_the_workspace():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = H.load_library()
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    assert lib.hps_leaf_maps_noalloc(0, None, 17, 0.25, 10.0, ctypes.c_void_p(dummy.data_ptr()), 1,
                                     ctypes.c_void_p(dummy.data_ptr())) == -1
