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

Nested Clenshaw-Curtis rules (Sec. 5: the adaptive scheme uses nested quadrature per refinement
level; Sec. 7 names Clenshaw-Curtis levels 2, 3, 4 with 5, 9, 17 points): level k has n = 2^k + 1
points x_j = cos(j pi / 2^k) (level 0: the single point 0), so every level's points are points of the
next. The tensor rule of level k in p dimensions has (2^k + 1)^p nodes; NestedCCSpace orders the
nodes of its finest level so that every coarser level's nodes are a prefix (by "birth level", the
coarsest level containing all coordinates of the node), and keeps each level's own weights.

Pinned by: tests/test_oracle_basis.py (count formula, orthonormality, recurrence against numpy's
Legendre series, Gauss exactness; Clenshaw-Curtis exactness, positivity, nesting and the printed
point counts).
"""
import itertools
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


# ------------------------------------------------------------------------------------------------
# nested Clenshaw-Curtis rules (adaptive quadrature per refinement level, Sec. 5 and Sec. 7)
# ------------------------------------------------------------------------------------------------
def clenshaw_curtis_1d(level: int):
    """Clenshaw-Curtis rule of the given level on [-1, 1]: 2^level + 1 points x_j = cos(j pi / 2^level),
    in ascending order, weights summing to 2 (level 0: the midpoint rule, 0 with weight 2). Weights by
    the closed form of Clenshaw and Curtis (1960) for an even number n = 2^level of intervals:
    w_0 = w_n = 1/(n^2 - 1); w_j = (2/n) [1 - sum_{k=1}^{n/2-1} 2 cos(2 k theta_j)/(4k^2 - 1)
    - cos(n theta_j)/(n^2 - 1)], theta_j = j pi / n."""
    if level == 0:
        return np.array([0.0]), np.array([2.0])
    n = 2 ** level
    j = np.arange(n + 1)
    theta = np.pi * j / n
    x = np.cos(theta)
    x[n // 2] = 0.0                        # cos(pi/2) exactly, so the rules nest bit for bit
    x[n // 2 + 1:] = -x[:n // 2][::-1]     # and the rule is exactly symmetric
    w = np.empty(n + 1)
    inner = np.ones(n - 1)
    for k in range(1, n // 2):
        inner -= 2.0 * np.cos(2 * k * theta[1:-1]) / (4 * k * k - 1)
    inner -= np.cos(n * theta[1:-1]) / (n * n - 1)
    w[1:-1] = 2.0 * inner / n
    w[0] = w[n] = 1.0 / (n * n - 1)
    return x[::-1].copy(), w[::-1].copy()


def cc_birth_level(j: int, kmax: int) -> int:
    """Coarsest level whose rule contains point j (ascending index 0..2^kmax) of the level-kmax rule."""
    n = 2 ** kmax
    if kmax == 0 or 2 * j == n:
        return 0
    if j == 0 or j == n:
        return 1
    tz = 0
    while j % 2 == 0:
        j //= 2
        tz += 1
    return kmax - tz


def nested_cc_tensor(p: int, kmax: int):
    """Tensor Clenshaw-Curtis nodes of level kmax on [-1,1]^p, ordered by birth level (the largest birth
    level of the node's coordinates), then by the coordinate indices (first dimension slowest), so that
    the nodes of every level k <= kmax are the first (2^k + 1)^p. Returns nodes (Q, p), birth (Q,) and
    [w_0, ..., w_kmax]: w_k (Q_k,) the tensor weights of level k at those first nodes, density 2^-p
    folded in (each sums to 1)."""
    x, _ = clenshaw_curtis_1d(kmax)
    n1 = x.size
    b1 = [cc_birth_level(j, kmax) for j in range(n1)]
    tuples = sorted(itertools.product(range(n1), repeat=p), key=lambda t: (max(b1[d] for d in t), t))
    nodes = np.array([[x[d] for d in t] for t in tuples]).reshape(-1, p)
    birth = np.array([max(b1[d] for d in t) for t in tuples], dtype=np.int64)
    weights = []
    for k in range(kmax + 1):
        xk, wk = clenshaw_curtis_1d(k)
        step = 2 ** (kmax - k)
        Qk = int(np.sum(birth <= k))
        wt = np.empty(Qk)
        for q in range(Qk):
            t = tuples[q]
            # coordinate index j of level kmax is index j / 2^(kmax-k) of level k (level 0: the midpoint)
            wt[q] = np.prod([wk[0] if k == 0 else wk[t[d] // step] for d in range(p)]) / 2.0 ** p
        weights.append(wt)
    return nodes, birth, weights


class NestedCCSpace:
    """Basis of total degree M with the nested tensor Clenshaw-Curtis rule of level kmax; level(k, n)
    views the first n basis functions with the level-k rule (its nodes are a prefix of this space's).
    The space itself behaves like StochasticSpace with the finest rule."""

    def __init__(self, p: int, M: int, kmax: int):
        self.p, self.M, self.kmax = p, M, kmax
        self.indices = total_degree_indices(p, M)
        self.N = self.indices.shape[0]
        self.nodes, self.birth, self.level_w = nested_cc_tensor(p, kmax)
        self.w = self.level_w[kmax]
        self.Q = self.w.shape[0]
        self.Phi = basis_table(self.indices, self.nodes)

    def level_q(self, k: int) -> int:
        return self.level_w[k].shape[0]

    def level(self, k: int, n: int):
        return _LevelView(self, k, n)

    def project(self, values_at_nodes: np.ndarray) -> np.ndarray:
        return np.einsum("k,...ka,ki->...ia", self.w, values_at_nodes, self.Phi)

    def evaluate(self, coeffs: np.ndarray) -> np.ndarray:
        return np.einsum("ki,...ia->...ka", self.Phi, coeffs)


class _LevelView:
    """The first n basis functions with the level-k nodes and weights of a NestedCCSpace."""

    def __init__(self, space: NestedCCSpace, k: int, n: int):
        self.N = n
        self.Q = space.level_q(k)
        self.w = space.level_w[k]
        self.nodes = space.nodes[:self.Q]
        self.Phi = space.Phi[:self.Q, :n]

    def project(self, values_at_nodes):
        return np.einsum("k,...ka,ki->...ia", self.w, values_at_nodes, self.Phi)

    def evaluate(self, coeffs):
        return np.einsum("ki,...ia->...ka", self.Phi, coeffs)
