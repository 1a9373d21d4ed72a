"""Host logic of the batched runner, on the CPU.

The library contexts are replaced by stand-ins with the same calls (a "solution" row echoes
the first impedance value of its right-hand side) and torch.cuda by a stand-in.  Checked:
problems run in waves of `slots`, one batched leaf build per wave over that wave's contexts,
a slot's mesh is rebuilt only when the shape changes, results come back in problem order with
each problem's own right-hand sides, and an error in one problem is raised after its wave.
"""
import contextlib

import numpy as np
import pytest

from paper_2511_00735_gb300 import batch as B
from paper_2511_00735_gb300 import inputs


class _FakeCuda:
    def Stream(self, device=0):
        return object()

    def stream(self, s):
        return contextlib.nullcontext()


class _FakeTorch:
    cuda = _FakeCuda()


class _FakeSolver:
    log = []
    fail_kappa = None

    def __init__(self, device, stream=None):
        self.id = len([e for e in _FakeSolver.log if e[0] == "new"])
        _FakeSolver.log.append(("new", self.id))

    def mesh(self, nx, N):
        self.nx, self.N, self.n_bdry = nx, N, 4 * nx * (N - 1)
        _FakeSolver.log.append(("mesh", self.id, nx, N))

    def node_coords(self):
        E, n = self.nx * self.nx, (self.N + 1) ** 2
        return np.zeros((E, n)), np.zeros((E, n))

    def set_coeff(self, kappa, b, eta=None):
        self.kappa = kappa

    def boundary_points(self):
        n = self.n_bdry
        return np.linspace(0.0, 1.0, n), np.zeros(n), np.zeros(n), -np.ones(n)

    def merge_levels(self, L_exact, exact_coarse=False):
        pass

    def gmres_solve(self, t, tol=1e-10, inner_iters=5, restart=60, max_outer=20, raise_on_notconv=True):
        if self.kappa == _FakeSolver.fail_kappa:
            raise RuntimeError("device error")
        return np.repeat(t[:, :1], 2, axis=1), {"rel_residual": [1e-11] * t.shape[0], "kappa": self.kappa}

    def close(self):
        pass


def _fake_build_leaves_batch(solvers, precision):
    _FakeSolver.log.append(("leaves", tuple(s.id for s in solvers)))


@pytest.fixture
def fake(monkeypatch):
    monkeypatch.setattr(B.H, "Solver", _FakeSolver)
    monkeypatch.setattr(B.H, "build_leaves_batch", _fake_build_leaves_batch)
    _FakeSolver.log, _FakeSolver.fail_kappa = [], None


def _problems():
    shapes = [(4, 8), (4, 8), (8, 8), (4, 8), (8, 12), (8, 12), (4, 8)]
    return [inputs.single_bump(nx, N, 10.0 + i, 1 + i % 3, seed=70 + i, L_exact=2) for i, (nx, N) in enumerate(shapes)]


def test_waves_meshes_and_order(fake):
    probs = _problems()
    br = B.BatchRunner(0, slots=3, torch_module=_FakeTorch())
    res = br.run(probs)
    br.close()
    leaves = [e[1] for e in _FakeSolver.log if e[0] == "leaves"]
    assert leaves == [(0, 1, 2), (0, 1, 2), (0,)]
    meshes = [e[1:] for e in _FakeSolver.log if e[0] == "mesh"]
    # slot 0: (4,8) then (4,8) again (kept), then (4,8) (kept); slot 1: (4,8) -> (8,12); slot 2: (8,8) -> (8,12)
    assert meshes == [(0, 4, 8), (1, 4, 8), (2, 8, 8), (1, 8, 12), (2, 8, 12)]
    for p, (g, info) in zip(probs, res):
        assert info["kappa"] == p.kappa and g.shape == (p.nrhs, 2)
        n = 4 * p.nx * (p.N - 1)
        bx, by, bnx, bny = np.linspace(0.0, 1.0, n), np.zeros(n), np.zeros(n), -np.ones(n)
        want = [inputs.plane_wave_impedance(th, p.kappa, p.eta, bx, by, bnx, bny)[0] for th in p.thetas]
        np.testing.assert_array_equal(g[:, 0], want)


def test_error_is_raised_after_its_wave(fake):
    probs = _problems()
    _FakeSolver.fail_kappa = probs[4].kappa
    br = B.BatchRunner(0, slots=3, torch_module=_FakeTorch())
    with pytest.raises(RuntimeError, match="device error"):
        br.run(probs)
    # the failing wave (problems 3-5) finished its leaves; the next wave never started
    leaves = [e[1] for e in _FakeSolver.log if e[0] == "leaves"]
    assert leaves == [(0, 1, 2), (0, 1, 2)]
