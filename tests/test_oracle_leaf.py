"""Pins of the oracle's leaf ItI map (section 3.1, eq. ItIOperator)."""
import math

import numpy as np
import pytest

from oracle import leaf as leafmod
from oracle.gll import gll_rule
from oracle.leaf import element_operators, index_sets, leaf_itI
from paper_2511_00735_gb300 import inputs


def _traces(N, h, kappa, eta, theta, x0=0.3, y0=0.2):
    """Exact incoming/outgoing impedance traces of a plane wave on an element's edge nodes."""
    xi, _ = gll_rule(N)
    t = x0 + (xi[1:-1] + 1) * h / 2, y0 + (xi[1:-1] + 1) * h / 2
    pts = [  # side, x, y, normal
        (np.full(N - 1, x0), t[1], (-1, 0)), (np.full(N - 1, x0 + h), t[1], (1, 0)),
        (t[0], np.full(N - 1, y0), (0, -1)), (t[0], np.full(N - 1, y0 + h), (0, 1)),
    ]
    fin, fout = [], []
    for x, y, n in pts:
        fin.append(inputs.plane_wave_impedance(theta, kappa, eta, x, y, *n))
        fout.append(inputs.plane_wave_impedance(theta, kappa, -eta, x, y, *n))
    return np.concatenate(fin), np.concatenate(fout)


def test_T_equals_identity_minus_2ieta_Y():
    # T = I_o Y and I_i Y = I on iota_Gamma give T = I - 2 i eta Y(iota_Gamma, :)
    N, h, eta = 10, 0.25, 7.0
    c = 49.0 * (1 - 0.3 * np.random.default_rng(0).random((N + 1) ** 2))
    out = leaf_itI(N, h, c, eta)
    Yg = out["Y"][index_sets(N)["gamma"]]
    np.testing.assert_allclose(out["T"], np.eye(4 * (N - 1)) - 2j * eta * Yg, atol=1e-12)


def test_corner_layouts_agree():
    N, h, eta = 8, 0.25, 10.0
    c = 100.0 * (1 - 0.5 * np.random.default_rng(1).random((N + 1) ** 2))
    T1 = leaf_itI(N, h, c, eta, corners="identity")["T"]
    T2 = leaf_itI(N, h, c, eta, corners="drop")["T"]
    np.testing.assert_allclose(T1, T2, atol=1e-13)


@pytest.mark.parametrize("N,kh,tol", [(8, 0.5, 1e-9), (12, 2.5, 1e-9), (16, 2.5, 1e-11)])
def test_plane_wave_consistency(N, kh, tol):
    # exact plane-wave traces: T f_in = f_out up to the discretisation error
    h = 0.25
    kappa = kh / h
    c = np.full((N + 1) ** 2, kappa ** 2)
    T = leaf_itI(N, h, c, kappa)["T"]
    fin, fout = _traces(N, h, kappa, kappa, 0.9)
    err = np.linalg.norm(T @ fin - fout) / np.linalg.norm(fout)
    assert err < tol, err


def test_plane_wave_spectral_convergence():
    h, kappa = 0.25, 10.0
    errs = []
    for N in (4, 6, 8, 10, 12):
        c = np.full((N + 1) ** 2, kappa ** 2)
        T = leaf_itI(N, h, c, kappa)["T"]
        fin, fout = _traces(N, h, kappa, kappa, 2.1)
        errs.append(np.linalg.norm(T @ fin - fout) / np.linalg.norm(fout))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-9 and errs[0] > 1e-5


def test_plus_c_sign_fails_plane_wave(monkeypatch):
    # planted mistake: the printed "+ diag(c)" sign destroys plane-wave consistency
    N, h, kappa = 12, 0.25, 10.0
    orig = leafmod.element_operators

    def plus_sign(N_, h_, c_, eta_):
        return orig(N_, h_, -np.asarray(c_), eta_)

    monkeypatch.setattr(leafmod, "element_operators", plus_sign)
    c = np.full((N + 1) ** 2, kappa ** 2)
    T = leafmod.leaf_itI(N, h, c, kappa)["T"]
    fin, fout = _traces(N, h, kappa, kappa, 0.9)
    assert np.linalg.norm(T @ fin - fout) / np.linalg.norm(fout) > 1e-2


def test_real_eta_without_i_fails():
    # planted mistake: impedance operators with a real eta term (the printed form)
    N, h, kappa = 12, 0.25, 10.0
    c = np.full((N + 1) ** 2, kappa ** 2)
    Lt, Dn, _, _, s = element_operators(N, h, c, kappa)
    Ig = np.eye((N + 1) ** 2)[s["gamma"]]
    L = Lt.astype(complex)
    L[s["gamma"]] = Dn + kappa * Ig
    for cn in s["corners"]:
        L[cn] = 0
        L[cn, cn] = 1
    T = (Dn - kappa * Ig) @ np.linalg.solve(L, np.eye((N + 1) ** 2)[:, s["gamma"]])
    fin, fout = _traces(N, h, kappa, kappa, 0.9)
    assert np.linalg.norm(T @ fin - fout) / np.linalg.norm(fout) > 1e-2


@pytest.mark.parametrize("kh", [0.5, 2.5])
def test_energy_and_unimodular_eigenvalues(kh):
    # b = 0: the ItI map conserves the edge-weighted energy of plane-wave traces (to 1e-12 at
    # N = 16) and its eigenvalues lie on the unit circle up to discretisation error; it is not
    # unitary as an operator (the edge-weighted singular values spread over [0.75, 1.35]),
    # reading A10
    N, h = 16, 0.25
    kappa = kh / h
    _, w = gll_rule(N)
    W = np.tile(w[1:-1] * h / 2, 4)
    c = np.full((N + 1) ** 2, kappa ** 2)
    T = leaf_itI(N, h, c, kappa)["T"]
    for th in (0.3, 1.7, 4.0):
        fin, _ = _traces(N, h, kappa, kappa, th)
        ein = np.sqrt(np.sum(W * abs(fin) ** 2))
        eout = np.sqrt(np.sum(W * abs(T @ fin) ** 2))
        assert abs(eout / ein - 1) < 1e-12
    ev = np.linalg.eigvals(T)
    assert np.all(abs(abs(ev) - 1) < 1e-2)


def test_manufactured_source_weighting():
    # reading A7: with b~ = w_i w_j s and s = kappa^2 b u_pw, the element solution with
    # incoming data I_i u_pw is u_pw (b != 0), up to discretisation error
    N, h, kappa, theta = 14, 0.25, 8.0, 0.6
    x0, y0 = 0.25, 0.5
    xi, w = gll_rule(N)
    xs = x0 + (xi + 1) * h / 2
    ys = y0 + (xi + 1) * h / 2
    X, Y = np.repeat(xs, N + 1), np.tile(ys, N + 1)
    bump = [inputs.Bump(1.2, 0.4, 0.6, 30.0)]
    b = inputs.eval_b(bump, X, Y)
    c = kappa ** 2 * (1 - b)
    upw = inputs.plane_wave(theta, kappa, X, Y)
    s = kappa ** 2 * b * upw
    btilde = np.kron(w * h / 2, w * h / 2) * s
    fin, fout = _traces(N, h, kappa, kappa, theta, x0, y0)
    u = leafmod.leaf_solution(N, h, c, kappa, fin, btilde)
    idx = [k for k in range((N + 1) ** 2) if k not in index_sets(N)["corners"]]
    err = np.linalg.norm(u[idx] - upw[idx]) / np.linalg.norm(upw[idx])
    assert err < 1e-9, err
    # and the closed impedance relation I_o u = T I_i u + H
    out = leaf_itI(N, h, c, kappa, btilde=btilde)
    np.testing.assert_allclose(out["T"] @ fin + out["H"], fout, atol=1e-7 * np.abs(fout).max())


# ---------------------------------------------------------------- corner post-processing
@pytest.mark.parametrize("N", [4, 8, 16])
def test_corner_values_exact_for_low_degree_edges(N):
    # edge restrictions of degree <= N-2 are extrapolated exactly (closed form)
    from oracle.gll import gll_rule
    from oracle.leaf import corner_values, index_sets, node

    xi, _ = gll_rule(N)
    X = np.repeat(xi, N + 1)
    Y = np.tile(xi, N + 1)
    d = N - 2
    u = (1 + 0.5j) * X ** d * Y ** (d // 2) - 2.0 * Y ** d + 0.3j * X * Y + 1.0
    v = u.copy()
    for k in index_sets(N)["corners"]:
        v[k] = 99.0
    w = corner_values(N, v)
    for i, j in ((0, 0), (0, N), (N, 0), (N, N)):
        assert abs(w[node(N, i, j)] - u[node(N, i, j)]) < 1e-11
    assert np.array_equal(np.delete(w, index_sets(N)["corners"]), np.delete(u, index_sets(N)["corners"]))


def test_corner_values_of_a_plane_wave_converge_spectrally():
    from oracle.gll import gll_rule
    from oracle.leaf import corner_values, index_sets

    errs = []
    for N in (8, 12, 16):
        xi, _ = gll_rule(N)
        X = np.repeat(xi, N + 1)
        Y = np.tile(xi, N + 1)
        u = np.exp(1j * 1.2 * (0.6 * X + 0.8 * Y))  # kappa h / 2 = 1.2
        c = index_sets(N)["corners"]
        v = u.copy()
        v[c] = 0.0
        errs.append(np.max(np.abs(corner_values(N, v)[c] - u[c])))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-9, errs


def test_corner_values_take_each_edge_to_its_own_end():
    # u = x + 2y is linear along every edge: each corner must get its own value; an
    # extrapolation taken to the wrong end of an edge (a swapped weight vector) is off by O(1)
    from oracle.gll import gll_rule
    from oracle.leaf import corner_values, node

    N = 8
    xi, _ = gll_rule(N)
    X = np.repeat(xi, N + 1)
    Y = np.tile(xi, N + 1)
    u = X + 2.0 * Y + 0.0j
    w = corner_values(N, u)
    for i, j, val in ((0, 0, -3.0), (0, N, 1.0), (N, 0, -1.0), (N, N, 3.0)):
        assert abs(w[node(N, i, j)] - val) < 1e-12, (i, j)
