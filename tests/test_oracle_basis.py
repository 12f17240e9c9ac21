"""Pins of oracle.basis against closed forms and library routines (Sec. 2, Sec. 3.1)."""
import itertools
from math import comb

import numpy as np
import pytest

from oracle import basis


@pytest.mark.parametrize("p,M", [(1, 5), (2, 4), (3, 5), (3, 6), (2, 9), (3, 2)])
def test_count_matches_binomial_and_brute_force(p, M):
    idx = basis.total_degree_indices(p, M)
    brute = {t for t in itertools.product(range(M + 1), repeat=p) if sum(t) <= M}
    assert basis.num_moments(p, M) == comb(M + p, p) == len(brute) == idx.shape[0]
    assert {tuple(r) for r in idx} == brute


def test_paper_counts():
    # N = 55 for total degree 9 in 2 uncertain dims (Sec. 7.2); 56 / 84 / 15 / 10 for the workloads
    assert basis.num_moments(2, 9) == 55
    assert basis.num_moments(3, 5) == 56
    assert basis.num_moments(3, 6) == 84
    assert basis.num_moments(2, 4) == 15
    assert basis.num_moments(3, 2) == 10


def test_graded_order():
    idx = basis.total_degree_indices(3, 4)
    deg = idx.sum(axis=1)
    assert np.all(np.diff(deg) >= 0)
    assert tuple(idx[0]) == (0, 0, 0)
    assert [tuple(r) for r in idx[1:4]] == [(1, 0, 0), (0, 1, 0), (0, 0, 1)]


@pytest.mark.parametrize("n", range(0, 12))
def test_legendre_recurrence_matches_numpy_series(n):
    x = np.linspace(-1, 1, 37)
    c = np.zeros(n + 1)
    c[n] = 1.0
    ref = np.sqrt(2 * n + 1) * np.polynomial.legendre.legval(x, c)
    np.testing.assert_allclose(basis.legendre_orthonormal(n, x), ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("n", [1, 2, 5, 10, 17])
def test_gauss_exactness_1d(n):
    nodes, w = basis.gauss_legendre_tensor(1, n)
    assert abs(w.sum() - 1.0) < 1e-15
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 1.0 / (k + 1)     # int_{-1}^{1} x^k dx / 2
        assert abs(np.sum(w * nodes[:, 0] ** k) - exact) < 1e-14


@pytest.mark.parametrize("p,M,nq", [(1, 5, 10), (3, 5, 6), (2, 4, 5), (3, 6, 7), (3, 2, 3)])
def test_orthonormality(p, M, nq):
    sp = basis.StochasticSpace(p, M, nq)
    G = sp.Phi.T @ (sp.w[:, None] * sp.Phi)
    np.testing.assert_allclose(G, np.eye(sp.N), atol=2e-14)
    assert sp.Q == nq ** p


def test_tensor_weights_are_products():
    sp = basis.StochasticSpace(2, 3, 4)
    x1, w1 = np.polynomial.legendre.leggauss(4)
    for k in range(sp.Q):
        a, b = divmod(k, 4)
        assert sp.nodes[k, 0] == x1[a] and sp.nodes[k, 1] == x1[b]
        assert abs(sp.w[k] - w1[a] * w1[b] / 4) < 1e-16
