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

void build_tables(int p, int M, int nq, HostTables& t) {
  t.p = p;
  t.M = M;
  t.indices.clear();
  std::vector<int> cur(p, 0);
  for (int deg = 0; deg <= M; ++deg) enumerate_degree(p, deg, 0, cur, t.indices);
  t.N = static_cast<int>(t.indices.size()) / p;

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

}  // namespace ipm
