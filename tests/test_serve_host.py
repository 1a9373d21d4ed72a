"""Host logic of the continuous-batching server, on the CPU.

The library context is replaced by a stand-in with the same calls (its "solution" row r
echoes the first impedance value of right-hand side r, so every result can be traced to
the request that asked for it) and torch.cuda by a stand-in that holds no memory.  Checked:
requests that arrive while their tree is busy join its next solve; different trees run
side by side; each request gets its own right-hand sides back; the HBM cap admits a new
tree only after evicting the least recently used idle one; a failing solve is reported on
its requests and the server keeps serving.
"""
import contextlib
import threading
import time

import numpy as np
import pytest

from paper_2511_00735_gb300 import inputs
from paper_2511_00735_gb300 import serve as S


class _FakeCuda:
    def empty_cache(self):
        pass

    def memory_reserved(self, device=0):
        return 0

    def Stream(self, device=0):
        return object()

    def stream(self, s):
        return contextlib.nullcontext()


class _FakeTorch:
    cuda = _FakeCuda()


class _FakeSolver:
    tree_bytes = 60_000_000
    gate = None            # threading.Event holding every solve until set
    fail_kappa = None      # solves of this wavenumber raise
    calls = []             # (kappa, number of right-hand sides) per solve call
    lock = threading.Lock()

    def __init__(self, device, stream=None):
        self.closed = False

    def mesh(self, nx, N):
        self.nx, self.N = nx, N
        self.n_bdry = 4 * nx * (N - 1)

    def node_coords(self):
        E, n = self.nx * self.nx, (self.N + 1) ** 2
        return np.zeros((E, n)), np.zeros((E, n))

    def set_coeff(self, kappa, b, eta=None):
        self.kappa = kappa

    def build_leaves(self, precision):
        pass

    def merge_levels(self, L_exact, exact_coarse=False):
        pass

    def boundary_points(self):
        n = self.n_bdry
        return np.linspace(0.0, 1.0, n), np.zeros(n), np.zeros(n), -np.ones(n)

    def bytes_held(self):
        return self.tree_bytes

    def gmres_solve(self, t, tol=1e-10, inner_iters=5, restart=60, max_outer=20, raise_on_notconv=True):
        if _FakeSolver.gate is not None:
            assert _FakeSolver.gate.wait(10.0)
        with _FakeSolver.lock:
            _FakeSolver.calls.append((self.kappa, t.shape[0]))
        if self.kappa == _FakeSolver.fail_kappa:
            raise RuntimeError("device error")
        g = np.repeat(t[:, :1], 3, axis=1)
        return g, {"iterations": [7] * t.shape[0], "rel_residual": [1e-11] * t.shape[0]}

    def release_workspace(self):
        pass

    def close(self):
        self.closed = True


@pytest.fixture
def fake(monkeypatch):
    monkeypatch.setattr(S.H, "Solver", _FakeSolver)
    _FakeSolver.gate, _FakeSolver.fail_kappa, _FakeSolver.calls = None, None, []
    yield
    _FakeSolver.gate = None


def _req(rid, base, thetas, arrival=0.0):
    p = inputs.Problem(nx=base.nx, N=base.N, kappa=base.kappa, eta=base.eta, bumps=base.bumps,
                       thetas=list(thetas), L_exact=base.L_exact, inner_iters=base.inner_iters, name=base.name)
    return S.Request(rid, p, arrival)


def _expected_first_values(req):
    n = 4 * req.prob.nx * (req.prob.N - 1)
    bx, by, bnx, bny = np.linspace(0.0, 1.0, n), np.zeros(n), np.zeros(n), -np.ones(n)
    return np.array([inputs.plane_wave_impedance(th, req.prob.kappa, req.prob.eta, bx, by, bnx, bny)[0]
                     for th in req.prob.thetas])


def _server(**kw):
    srv = S.Server(device=0, torch_module=_FakeTorch(), **kw)
    srv.t_origin = time.perf_counter()
    return srv


def _wait(cond, timeout=10.0):
    t0 = time.perf_counter()
    while not cond():
        assert time.perf_counter() - t0 < timeout
        time.sleep(0.005)


def test_busy_tree_batches_late_requests(fake):
    k1 = inputs.single_bump(4, 8, 10.0, 1, seed=41, L_exact=2)
    k2 = inputs.single_bump(4, 8, 12.0, 1, seed=42, L_exact=2)
    _FakeSolver.gate = threading.Event()
    srv = _server(workers=2, hbm_cap=1e12)
    try:
        a = _req(0, k1, [0.1, 0.2])
        srv.submit(a)
        _wait(lambda: any(t.busy for t in srv.trees.values()))
        b, c, d = _req(1, k1, [0.3]), _req(2, k1, [0.4, 0.5, 0.6]), _req(3, k2, [0.7])
        for r in (b, c, d):
            srv.submit(r)
        # the other worker takes the other tree while the first is busy
        _wait(lambda: len(srv.trees) == 2 and all(t.busy for t in srv.trees.values()))
        assert [r.rid for r in srv.pending] == [1, 2]
        _FakeSolver.gate.set()
        done = srv.drain(4, timeout=30.0)
    finally:
        srv.close()
    assert sorted(r.rid for r in done) == [0, 1, 2, 3]
    assert a.info["batched_with"] == 1 and d.info["batched_with"] == 1
    assert b.info["batched_with"] == 2 and c.info["batched_with"] == 2
    assert sorted(_FakeSolver.calls) == sorted([(10.0, 2), (10.0, 4), (12.0, 1)])
    for r in (a, b, c, d):
        assert r.g.shape == (r.prob.nrhs, 3)
        np.testing.assert_array_equal(r.g[:, 0], _expected_first_values(r))
        assert r.done >= r.arrival and max(r.info["rel_residual"]) <= srv.tol


def test_hbm_cap_evicts_least_recently_used_idle_tree(fake):
    keys = [inputs.single_bump(4, 8, 10.0 + i, 1, seed=50 + i, L_exact=2) for i in range(3)]
    need = S.tree_only_bytes(4, 8, S.H.HPS_MIXED) + S.krylov_bytes(4, 8, 1)
    cap = _FakeSolver.tree_bytes + need - 1  # one idle tree plus a new tree's job does not fit
    assert need <= cap
    srv = _server(workers=1, hbm_cap=cap)
    try:
        order = [0, 1, 1, 2, 0]
        for i, k in enumerate(order):
            srv.submit(_req(i, keys[k], [0.1 * (i + 1)]))
            srv.drain(i + 1, timeout=30.0)
        held_keys = [t.key for t in srv.trees.values()]
        evictions, peak = srv.evictions, srv.peak_bytes
    finally:
        srv.close()
    # a new tree evicts the idle one each time; a repeated key reuses its tree
    assert evictions == 3
    assert len(held_keys) == 1 and held_keys[0] == _req(0, keys[0], [0.0]).key
    assert peak <= cap
    assert [c[1] for c in _FakeSolver.calls] == [1, 1, 1, 1, 1]


def test_failed_solve_is_reported_and_server_continues(fake):
    bad = inputs.single_bump(4, 8, 10.0, 1, seed=61, L_exact=2)
    good = inputs.single_bump(4, 8, 11.0, 1, seed=62, L_exact=2)
    _FakeSolver.fail_kappa = 10.0
    srv = _server(workers=1, hbm_cap=1e12)
    try:
        r0, r1 = _req(0, bad, [0.1, 0.2]), _req(1, good, [0.3])
        srv.submit(r0)
        srv.submit(r1)
        done = srv.drain(2, timeout=30.0)
        busy = [t.busy for t in srv.trees.values()]
    finally:
        srv.close()
    assert len(done) == 2 and not any(busy)
    assert "error" in r0.info and r0.info["rel_residual"] == [float("inf")]
    assert "error" not in r1.info and max(r1.info["rel_residual"]) <= 1e-10
    np.testing.assert_array_equal(r1.g[:, 0], _expected_first_values(r1))
