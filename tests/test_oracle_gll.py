"""Pins of the oracle's GLL rule (section 3.1) against closed forms and exact identities."""
import math

import numpy as np
import pytest

from oracle.gll import element_1d, gll_diff, gll_rule


@pytest.mark.parametrize("N,nodes,weights", [
    # textbook closed forms (e.g. Abramowitz & Stegun 25.4.32; Canuto et al. table 2.3)
    (2, [-1.0, 0.0, 1.0], [1 / 3, 4 / 3, 1 / 3]),
    (3, [-1.0, -1 / math.sqrt(5), 1 / math.sqrt(5), 1.0], [1 / 6, 5 / 6, 5 / 6, 1 / 6]),
    (4, [-1.0, -math.sqrt(3 / 7), 0.0, math.sqrt(3 / 7), 1.0],
     [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]),
])
def test_closed_forms(N, nodes, weights):
    x, w = gll_rule(N)
    np.testing.assert_allclose(x, nodes, atol=1e-15)
    np.testing.assert_allclose(w, weights, atol=1e-15)


@pytest.mark.parametrize("N", [2, 5, 8, 12, 16, 20])
def test_quadrature_exact_to_degree_2N_minus_1(N):
    x, w = gll_rule(N)
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(2 * N):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 2e-14, k
    # degree 2N is NOT integrated exactly by an (N+1)-point Lobatto rule
    assert abs(np.dot(w, x ** (2 * N)) - 2.0 / (2 * N + 1)) > 1e-12


@pytest.mark.parametrize("N", [3, 8, 16])
def test_differentiation_exact_on_degree_N(N):
    x, _ = gll_rule(N)
    D = gll_diff(N, x)
    for k in range(N + 1):
        f = x ** k
        df = k * x ** (k - 1) if k > 0 else np.zeros_like(x)
        np.testing.assert_allclose(D @ f, df, atol=1e-11 * max(1, k * k))


@pytest.mark.parametrize("N", [4, 8, 16])
def test_summation_by_parts(N):
    x, w = gll_rule(N)
    D = gll_diff(N, x)
    M = np.diag(w)
    B = np.zeros((N + 1, N + 1))
    B[0, 0], B[N, N] = -1.0, 1.0
    np.testing.assert_allclose(M @ D + D.T @ M, B, atol=1e-13)


def test_element_scaling():
    # K = D^T M D is h-invariant and M scales with h/2 (reading A8)
    _, w1, D1, M1, K1 = element_1d(8, 1.0)
    _, w2, D2, M2, K2 = element_1d(8, 0.25)
    np.testing.assert_allclose(K1 / 1.0, K2 * 0.25, rtol=1e-13)
    np.testing.assert_allclose(w2, w1 * 0.25, rtol=1e-15)
