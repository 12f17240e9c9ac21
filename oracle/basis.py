"""gPC basis and quadrature (test infrastructure; see ``oracle/__init__``).

* Multi-indices with total degree |i| = i_1 + ... + i_p <= M; there are N = C(M+p, p) of them
  (Sec. 2, Eq. numberBasisFcts).
* Orthonormal basis for xi ~ U[-1,1]^p: phi_i(xi) = prod_n sqrt(2 i_n + 1) P_{i_n}(xi_n), so that
  <phi_i phi_j> = delta_ij under the density f = 2^-p (Sec. 2 below Eq. numberBasisFcts; App. A names
  the Legendre polynomials for the uniform case).
* Quadrature <h>_Q = sum_k w_k h(xi_k) f(xi_k) (Sec. 3.1): tensor Gauss-Legendre rules. The weights
  returned here already include f, so they sum to 1.

Ordering of the multi-indices ("graded"): ascending total degree; within one degree, descending
lexicographic order of (i_1, ..., i_p), e.g. for p = 3, degree 1: (1,0,0), (0,1,0), (0,0,1).
This is the moment order of every [cell][moment][variable] array.

Pinned by: tests/test_oracle_basis.py (count formula, orthonormality, recurrence against numpy's
Legendre series, Gauss exactness).
"""
from math import comb

import numpy as np


def num_moments(p: int, M: int) -> int:
    """N = C(M+p, p) (Sec. 2, Eq. numberBasisFcts)."""
    return comb(M + p, p)


def total_degree_indices(p: int, M: int) -> np.ndarray:
    """All multi-indices i in N^p with |i| <= M, in graded order. Shape (N, p)."""
    out = []
    for deg in range(M + 1):
        level = []

        def rec(prefix, remaining, dims_left):
            if dims_left == 1:
                level.append(tuple(prefix + [remaining]))
                return
            for k in range(remaining, -1, -1):
                rec(prefix + [k], remaining - k, dims_left - 1)

        rec([], deg, p)
        out.extend(level)
    return np.array(out, dtype=np.int64).reshape(-1, p)


def legendre_orthonormal(n: int, x: np.ndarray) -> np.ndarray:
    """sqrt(2n+1) P_n(x) via the three-term recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}."""
    x = np.asarray(x, dtype=np.float64)
    p_prev = np.ones_like(x)
    if n == 0:
        return p_prev
    p_cur = x.copy()
    for k in range(1, n):
        p_prev, p_cur = p_cur, ((2 * k + 1) * x * p_cur - k * p_prev) / (k + 1)
    return np.sqrt(2 * n + 1) * p_cur


def gauss_legendre_tensor(p: int, n: int):
    """Tensor Gauss-Legendre rule with n nodes per dimension on [-1,1]^p.

    Returns nodes (Q, p) and weights (Q,) with the density f = 2^-p folded in (sum = 1).
    Node order: the last dimension runs fastest.
    """
    x1, w1 = np.polynomial.legendre.leggauss(n)
    grids = np.meshgrid(*([x1] * p), indexing="ij")
    wgrids = np.meshgrid(*([w1] * p), indexing="ij")
    nodes = np.stack([g.reshape(-1) for g in grids], axis=1)
    weights = np.prod(np.stack([g.reshape(-1) for g in wgrids], axis=1), axis=1) / (2.0 ** p)
    return nodes, weights


def basis_table(indices: np.ndarray, nodes: np.ndarray) -> np.ndarray:
    """Phi[k, i] = phi_i(xi_k), shape (Q, N)."""
    Q = nodes.shape[0]
    N, p = indices.shape
    Phi = np.ones((Q, N))
    for i in range(N):
        for d in range(p):
            Phi[:, i] *= legendre_orthonormal(int(indices[i, d]), nodes[:, d])
    return Phi


class StochasticSpace:
    """Basis + quadrature of one problem: p uncertain dims, total degree M, n_q nodes per dim."""

    def __init__(self, p: int, M: int, n_q: int):
        self.p, self.M, self.n_q = p, M, n_q
        self.indices = total_degree_indices(p, M)
        self.N = self.indices.shape[0]
        self.nodes, self.w = gauss_legendre_tensor(p, n_q)
        self.Q = self.w.shape[0]
        self.Phi = basis_table(self.indices, self.nodes)

    def project(self, values_at_nodes: np.ndarray) -> np.ndarray:
        """<v phi^T>_Q^T for v given at the nodes: (..., Q, m) -> (..., N, m)."""
        return np.einsum("k,...ka,ki->...ia", self.w, values_at_nodes, self.Phi)

    def evaluate(self, coeffs: np.ndarray) -> np.ndarray:
        """coeffs^T phi(xi_k) at every node: (..., N, m) -> (..., Q, m)."""
        return np.einsum("ki,...ia->...ka", self.Phi, coeffs)
