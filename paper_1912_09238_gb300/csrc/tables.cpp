// tables.cpp -- host construction of the gPC basis and quadrature tables.
//
// * Multi-indices of total degree <= M (Sec. 2, Eq. numberBasisFcts: N = C(M+p, p)), graded order:
//   ascending degree, then descending lexicographic order of (i_1, ..., i_p).
// * Orthonormal Legendre basis for xi ~ U[-1,1]^p (Sec. 2, <phi_i phi_j> = delta_ij; App. A names the
//   Legendre polynomials): phi_i(xi) = prod_n sqrt(2 i_n + 1) P_{i_n}(xi_n).
// * Tensor Gauss-Legendre quadrature <h>_Q = sum_k w_k h(xi_k) f(xi_k) (Sec. 3.1); the density
//   f = 2^-p is folded into the weights. 1-D nodes are the roots of P_n found by Newton's method on
//   the three-term recurrence, started from cos(pi (k - 1/4) / (n + 1/2)); weights
//   2 / ((1 - x^2) P_n'(x)^2).
// * Nested Clenshaw-Curtis rules (Sec. 5: nested quadrature per refinement level; Sec. 7: levels with
//   2^k + 1 points): points -cos(pi j / 2^k), ascending (level 0: the midpoint); the weights solve the
//   exactness conditions sum_j w_j T_m(x_j) = int_{-1}^{1} T_m for the Chebyshev polynomials
//   m = 0 .. 2^k (a dense solve in long double). Tensor nodes of the finest level are ordered by birth
//   level (the coarsest level containing every coordinate), then by their coordinate indices (first
//   dimension slowest), so that each level's nodes are a prefix; every level keeps its own weights.
#include <algorithm>
#include <array>
#include <cmath>
#include <vector>

#include "ipm_host.h"

namespace ipm {

static void legendre_and_derivative(int n, double x, double* pn, double* dpn) {
  double p0 = 1.0, p1 = x;
  if (n == 0) {
    *pn = 1.0;
    *dpn = 0.0;
    return;
  }
  for (int k = 1; k < n; ++k) {
    const double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  *pn = p1;
  *dpn = n * (x * p1 - p0) / (x * x - 1.0);
}

void gauss_legendre_1d(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int k = 1; k <= n; ++k) {
    double z = std::cos(pi * (k - 0.25) / (n + 0.5));
    double pn = 0.0, dpn = 1.0;
    for (int it = 0; it < 100; ++it) {
      legendre_and_derivative(n, z, &pn, &dpn);
      const double dz = pn / dpn;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    legendre_and_derivative(n, z, &pn, &dpn);
    // roots come out in descending order; store ascending
    x[n - k] = z;
    w[n - k] = 2.0 / ((1.0 - z * z) * dpn * dpn);
  }
}

static double legendre_orthonormal(int n, double x) {
  double p0 = 1.0, p1 = x;
  if (n == 0) return 1.0;
  for (int k = 1; k < n; ++k) {
    const double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  return std::sqrt(2.0 * n + 1.0) * p1;
}

static void enumerate_degree(int p, int remaining, int dim, std::vector<int>& cur, std::vector<int>& out) {
  if (dim == p - 1) {
    cur[dim] = remaining;
    out.insert(out.end(), cur.begin(), cur.end());
    return;
  }
  for (int k = remaining; k >= 0; --k) {
    cur[dim] = k;
    enumerate_degree(p, remaining - k, dim + 1, cur, out);
  }
}

static void basis_indices(int p, int M, HostTables& t) {
  t.p = p;
  t.M = M;
  t.indices.clear();
  std::vector<int> cur(p, 0);
  for (int deg = 0; deg <= M; ++deg) enumerate_degree(p, deg, 0, cur, t.indices);
  t.N = static_cast<int>(t.indices.size()) / p;
}

// Phi [Q][N], Phi^T [N][Q] and the moment pairs, from t.nodes and t.indices
static void basis_values(HostTables& t) {
  const int Q = t.Q, p = t.p;
  t.Phi.assign(static_cast<size_t>(Q) * t.N, 1.0);
  for (int k = 0; k < Q; ++k)
    for (int i = 0; i < t.N; ++i) {
      double v = 1.0;
      for (int d = 0; d < p; ++d)
        v *= legendre_orthonormal(t.indices[static_cast<size_t>(i) * p + d], t.nodes[static_cast<size_t>(k) * p + d]);
      t.Phi[static_cast<size_t>(k) * t.N + i] = v;
    }
  t.PhiT.assign(t.Phi.size(), 0.0);
  for (int k = 0; k < Q; ++k)
    for (int i = 0; i < t.N; ++i) t.PhiT[static_cast<size_t>(i) * Q + k] = t.Phi[static_cast<size_t>(k) * t.N + i];
  t.pairs.clear();
  for (int i = 0; i < t.N; ++i)
    for (int j = 0; j <= i; ++j) t.pairs.push_back((static_cast<uint32_t>(i) << 16) | static_cast<uint32_t>(j));
}

// Clenshaw-Curtis points of level k (ascending) and weights summing to 2
void clenshaw_curtis_1d(int k, std::vector<double>& x, std::vector<double>& w) {
  if (k == 0) {
    x.assign(1, 0.0);
    w.assign(1, 2.0);
    return;
  }
  const int n = 1 << k;
  const double pi = 3.14159265358979323846;
  x.assign(n + 1, 0.0);
  for (int a = 0; a < n / 2; ++a) {
    x[a] = -std::cos(pi * a / n);
    x[n - a] = -x[a];
  }
  // exactness on T_0 .. T_n: A w = b with A[m][j] = cos(m theta_j), theta_j = pi (n - j) / n (x_j = cos theta_j)
  const int n1 = n + 1;
  std::vector<long double> A(static_cast<size_t>(n1) * n1), b(n1);
  const long double pil = 3.14159265358979323846264338327950288L;
  for (int m = 0; m < n1; ++m) {
    for (int j = 0; j < n1; ++j) A[static_cast<size_t>(m) * n1 + j] = std::cos(pil * m * (n - j) / n);
    b[m] = (m % 2 == 0) ? 2.0L / (1.0L - static_cast<long double>(m) * m) : 0.0L;
  }
  for (int col = 0; col < n1; ++col) {           // Gaussian elimination with partial pivoting
    int piv = col;
    for (int r = col + 1; r < n1; ++r)
      if (std::fabs(A[static_cast<size_t>(r) * n1 + col]) > std::fabs(A[static_cast<size_t>(piv) * n1 + col])) piv = r;
    if (piv != col) {
      for (int c = 0; c < n1; ++c) std::swap(A[static_cast<size_t>(col) * n1 + c], A[static_cast<size_t>(piv) * n1 + c]);
      std::swap(b[col], b[piv]);
    }
    for (int r = col + 1; r < n1; ++r) {
      const long double f = A[static_cast<size_t>(r) * n1 + col] / A[static_cast<size_t>(col) * n1 + col];
      for (int c = col; c < n1; ++c) A[static_cast<size_t>(r) * n1 + c] -= f * A[static_cast<size_t>(col) * n1 + c];
      b[r] -= f * b[col];
    }
  }
  std::vector<long double> sol(n1);
  for (int r = n1 - 1; r >= 0; --r) {
    long double v = b[r];
    for (int c = r + 1; c < n1; ++c) v -= A[static_cast<size_t>(r) * n1 + c] * sol[c];
    sol[r] = v / A[static_cast<size_t>(r) * n1 + r];
  }
  w.assign(n1, 0.0);
  for (int j = 0; j < n1; ++j) w[j] = static_cast<double>(sol[j]);
}

static int cc_birth(int j, int kmax) {
  const int n = 1 << kmax;
  if (kmax == 0 || 2 * j == n) return 0;
  if (j == 0 || j == n) return 1;
  int tz = 0;
  while (j % 2 == 0) {
    j /= 2;
    ++tz;
  }
  return kmax - tz;
}

void build_tables_cc(int p, int M, int kmax, HostTables& t, std::vector<std::vector<double>>& level_w) {
  basis_indices(p, M, t);
  std::vector<double> x, wdummy;
  clenshaw_curtis_1d(kmax, x, wdummy);
  const int n1 = static_cast<int>(x.size());
  std::vector<int> b1(n1);
  for (int j = 0; j < n1; ++j) b1[j] = cc_birth(j, kmax);
  int Q = 1;
  for (int d = 0; d < p; ++d) Q *= n1;
  // (birth level, coordinate indices) of every tensor node, sorted
  std::vector<std::array<int, 4>> key(Q);
  for (int q = 0; q < Q; ++q) {
    int rem = q, birth = 0;
    std::array<int, 4> k4 = {0, 0, 0, 0};
    for (int d = p - 1; d >= 0; --d) {
      k4[1 + d] = rem % n1;
      rem /= n1;
      birth = std::max(birth, b1[k4[1 + d]]);
    }
    k4[0] = birth;
    key[q] = k4;
  }
  std::sort(key.begin(), key.end());
  t.Q = Q;
  t.nodes.assign(static_cast<size_t>(Q) * p, 0.0);
  for (int q = 0; q < Q; ++q)
    for (int d = 0; d < p; ++d) t.nodes[static_cast<size_t>(q) * p + d] = x[key[q][1 + d]];
  level_w.assign(kmax + 1, std::vector<double>());
  for (int k = 0; k <= kmax; ++k) {
    std::vector<double> xk, wk;
    clenshaw_curtis_1d(k, xk, wk);
    const int step = 1 << (kmax - k);
    int Qk = 0;
    while (Qk < Q && key[Qk][0] <= k) ++Qk;
    level_w[k].assign(Qk, 0.0);
    for (int q = 0; q < Qk; ++q) {
      double v = 1.0;
      for (int d = 0; d < p; ++d) v *= 0.5 * (k == 0 ? wk[0] : wk[key[q][1 + d] / step]);
      level_w[k][q] = v;
    }
  }
  t.w = level_w[kmax];
  basis_values(t);
}

void build_tables(int p, int M, int nq, HostTables& t) {
  basis_indices(p, M, t);

  std::vector<double> x1, w1;
  gauss_legendre_1d(nq, x1, w1);
  int Q = 1;
  for (int d = 0; d < p; ++d) Q *= nq;
  t.Q = Q;
  t.nodes.assign(static_cast<size_t>(Q) * p, 0.0);
  t.w.assign(Q, 0.0);
  for (int k = 0; k < Q; ++k) {
    int rem = k;
    double wk = 1.0;
    for (int d = p - 1; d >= 0; --d) {       // last dimension fastest
      const int a = rem % nq;
      rem /= nq;
      t.nodes[static_cast<size_t>(k) * p + d] = x1[a];
      wk *= 0.5 * w1[a];
    }
    t.w[k] = wk;
  }
  basis_values(t);
}

const char* cc_levels(const ipm_quadrature* quad, int M0, int n, int* out) {
  bool any = false;
  for (int l = 0; l < n; ++l) any = any || quad->cc_level[l] != 0;
  for (int l = 0; l < n; ++l) {
    const int M = M0 + l;
    int k = quad->cc_level[l];
    if (!any) {
      k = 1;
      while ((1 << k) + 1 < M + 2) ++k;
    }
    if (k < 0 || k > 6) return "Clenshaw-Curtis levels must lie in 0..6";
    const int points = k == 0 ? 1 : (1 << k) + 1;
    if (points < M + 1) return "a Clenshaw-Curtis level has fewer points per dimension than its degree + 1";
    if (l > 0 && k < out[l - 1]) return "Clenshaw-Curtis levels must not decrease with the refinement level";
    out[l] = k;
  }
  return nullptr;
}

}  // namespace ipm
