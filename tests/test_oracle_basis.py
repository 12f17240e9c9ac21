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


# ---------- nested Clenshaw-Curtis rules (Sec. 5 nested quadrature; Sec. 7 levels and counts) ----------
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_clenshaw_curtis_weights_solve_the_moment_equations(k):
    """Independent of the closed form: the weights that make the rule exact on P_0..P_n at the
    Chebyshev points (a Legendre Vandermonde solve) are the closed-form weights; all are positive."""
    x, w = basis.clenshaw_curtis_1d(k)
    n = x.size
    V = np.stack([np.polynomial.legendre.legval(x, np.eye(n)[d]) for d in range(n)])
    rhs = np.zeros(n)
    rhs[0] = 2.0
    assert np.abs(np.linalg.solve(V, rhs) - w).max() < 1e-13
    assert np.all(w > 0) and abs(w.sum() - 2.0) < 1e-14
    # odd point count: exact one degree beyond the interpolation degree, by symmetry
    assert abs(np.sum(w * x ** n) - (2.0 / (n + 1) if n % 2 == 0 else 0.0)) < 1e-14


def test_clenshaw_curtis_rules_are_nested():
    for k in range(5):
        a, _ = basis.clenshaw_curtis_1d(k)
        b, _ = basis.clenshaw_curtis_1d(k + 1)
        assert all(np.min(np.abs(b - v)) == 0.0 for v in a)


def test_paper_clenshaw_curtis_point_counts():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "clenshaw_curtis_points.txt")
    rows = [tuple(int(t) for t in line.split()) for line in open(path) if line.strip() and not line.startswith("#")]
    assert len(rows) == 6
    for p, k, count in rows:
        if p == 1:
            assert basis.clenshaw_curtis_1d(k)[0].size == count
        _, _, W = basis.nested_cc_tensor(p, k)
        assert W[k].size == count


@pytest.mark.parametrize("p,kmax", [(1, 3), (2, 3), (3, 2)])
def test_nested_tensor_levels_are_prefixes_with_their_own_weights(p, kmax):
    nodes, birth, W = basis.nested_cc_tensor(p, kmax)
    assert np.all(np.diff(birth) >= 0)
    for k in range(kmax + 1):
        x, w = basis.clenshaw_curtis_1d(k)
        Qk = W[k].size
        assert Qk == x.size ** p
        # the prefix is the level-k tensor grid, and its weights are the level-k tensor weights
        grid = {tuple(t): np.prod([w[list(x).index(c)] for c in t]) / 2 ** p
                for t in itertools.product(x, repeat=p)}
        got = {tuple(v): wt for v, wt in zip(nodes[:Qk], W[k])}
        assert set(got) == set(grid)
        assert max(abs(got[t] - grid[t]) for t in grid) < 1e-15
        # exact for tensor monomials of degree <= 2^k + 1 per dimension (degree 1 at level 0)
        top = 1 if k == 0 else x.size
        for e in itertools.product(range(top + 1), repeat=p):
            exact = np.prod([(1.0 / (d + 1) if d % 2 == 0 else 0.0) for d in e])
            assert abs(np.sum(W[k] * np.prod(nodes[:Qk] ** np.array(e), axis=1)) - exact) < 1e-14


def test_nested_space_is_orthonormal_where_the_rule_is_exact():
    sp = basis.NestedCCSpace(2, 4, 3)          # degree 8 per dimension needs 9 points: level 3
    G = sp.Phi.T @ (sp.w[:, None] * sp.Phi)
    assert np.abs(G - np.eye(sp.N)).max() < 1e-13
    lv = sp.level(2, 6)                        # degree 2 (6 functions) on the level-2 rule (5 points)
    G2 = lv.Phi.T @ (lv.w[:, None] * lv.Phi)
    assert np.abs(G2 - np.eye(6)).max() < 1e-13
