// ic.cuh -- the initial data at one quadrature node: exact cell averages of the uncertain initial
// states (Algorithm 1, first loop: u_j^0 = (1/dx) int_cell u_IC(x, xi_k) dx, before the projection
// onto the basis). The IPM initialisation projects them; the collocation solver keeps them node by
// node. Every parameter X of the data is X + sum_d dX[d] xi_d.
//   1-D Riemann data: frac U_L(xi) + (1 - frac) U_R(xi), frac = clip((x0(xi) - x_{j-1/2}) / dx, 0, 1).
//   2-D (Sec. 7): uniform freestream (Mach and flow angle uncertain); a shear band averaged exactly
//   over the cell's y-extent with the transverse velocity at the cell centre's x; a Riemann jump in x
//   (interface x0(xi)) averaged exactly over the cell's x-extent.
#pragma once
#include <cmath>

#include "../../include/ipm.h"

namespace ipm {

struct IC1D {
  double x_lo, dx, gamma;
  double x0, dx0[3];
  double left[4], dleft[4][3], right[4], dright[4][3];
};

struct IC2D {
  int nx, ny, ic_kind;
  double x_lo, dx, y_lo, dy, gamma;
  double x0, dx0[3];
  double left[4], dleft[4][3], right[4], dright[4][3];
  double param[4], dparam[4][3];
};

inline IC1D ic1d_params(const ipm_problem& prob) {
  IC1D a;
  a.x_lo = prob.x_lo;
  a.dx = (prob.x_hi - prob.x_lo) / prob.nx;
  a.gamma = prob.gamma;
  a.x0 = prob.ic_x0;
  for (int d = 0; d < 3; ++d) a.dx0[d] = prob.ic_dx0[d];
  for (int v = 0; v < 4; ++v) {
    a.left[v] = prob.ic_left[v];
    a.right[v] = prob.ic_right[v];
    for (int d = 0; d < 3; ++d) {
      a.dleft[v][d] = prob.ic_dleft[v][d];
      a.dright[v][d] = prob.ic_dright[v][d];
    }
  }
  return a;
}

inline IC2D ic2d_params(const ipm_problem& prob) {
  IC2D a;
  a.nx = prob.nx;
  a.ny = prob.ny;
  a.ic_kind = prob.ic_kind;
  a.x_lo = prob.x_lo;
  a.dx = (prob.x_hi - prob.x_lo) / prob.nx;
  a.y_lo = prob.y_lo;
  a.dy = (prob.y_hi - prob.y_lo) / prob.ny;
  a.gamma = prob.gamma;
  a.x0 = prob.ic_x0;
  for (int d = 0; d < 3; ++d) a.dx0[d] = prob.ic_dx0[d];
  for (int v = 0; v < 4; ++v) {
    a.left[v] = prob.ic_left[v];
    a.right[v] = prob.ic_right[v];
    a.param[v] = prob.ic_param[v];
    for (int d = 0; d < 3; ++d) {
      a.dleft[v][d] = prob.ic_dleft[v][d];
      a.dright[v][d] = prob.ic_dright[v][d];
      a.dparam[v][d] = prob.ic_dparam[v][d];
    }
  }
  return a;
}

#ifdef __CUDACC__
__device__ __forceinline__ double affine3(double v0, const double* d, const double* xi, int P) {
  double v = v0;
  for (int k = 0; k < P; ++k) v = fma(d[k], xi[k], v);
  return v;
}

// primitive (rho, v_1 .. v_D, p) -> conserved (rho, rho v, E); M = 1: the scalar itself
template <int M>
__device__ __forceinline__ void primitive_to_conserved(const double* prim, double gamma, double* u) {
  if (M == 1) {
    u[0] = prim[0];
  } else {
    constexpr int D = M - 2;
    const double rho = prim[0], p = prim[D + 1];
    double vsq = 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      u[1 + d] = rho * prim[1 + d];
      vsq = fma(prim[1 + d], prim[1 + d], vsq);
    }
    u[0] = rho;
    u[M - 1] = p / (gamma - 1.0) + 0.5 * rho * vsq;
  }
}

// cell j (ghost-inclusive index, cell j spans [x_lo + (j-1) dx, x_lo + j dx]) at node xi
template <int M>
__device__ __forceinline__ void ic1d_average(const IC1D& a, int j, const double* xi, int P, double* ub) {
  const double x_left = a.x_lo + (j - 1) * a.dx;
  double x0 = a.x0, pl[4], pr[4];
  for (int d = 0; d < P; ++d) x0 = fma(a.dx0[d], xi[d], x0);
  const int nprim = (M == 1) ? 1 : M;
  for (int v = 0; v < nprim; ++v) {
    pl[v] = a.left[v];
    pr[v] = a.right[v];
    for (int d = 0; d < P; ++d) {
      pl[v] = fma(a.dleft[v][d], xi[d], pl[v]);
      pr[v] = fma(a.dright[v][d], xi[d], pr[v]);
    }
  }
  double UL[M], UR[M];
  primitive_to_conserved<M>(pl, a.gamma, UL);
  primitive_to_conserved<M>(pr, a.gamma, UR);
  const double frac = fmin(fmax((x0 - x_left) / a.dx, 0.0), 1.0);
#pragma unroll
  for (int c = 0; c < M; ++c) ub[c] = frac * UL[c] + (1.0 - frac) * UR[c];
}

__device__ __forceinline__ void prim4_to_cons(double rho, double v1, double v2, double p, double g, double* u) {
  u[0] = rho;
  u[1] = rho * v1;
  u[2] = rho * v2;
  u[3] = p / (g - 1.0) + 0.5 * rho * (v1 * v1 + v2 * v2);
}

// 2-D cell at ghost-inclusive column ii and row jj, at node xi
__device__ __forceinline__ void ic2d_average(const IC2D& a, int ii, int jj, const double* xi, int P, double* ub) {
  const int nx = a.nx, ny = a.ny;
  if (a.ic_kind == IPM_IC_FREESTREAM) {
    const double rho = a.param[0], p = a.param[1];
    const double mach = affine3(a.param[2], a.dparam[2], xi, P);
    const double th = affine3(a.param[3], a.dparam[3], xi, P) * (M_PI / 180.0);
    const double cs = sqrt(a.gamma * p / rho);
    prim4_to_cons(rho, mach * cs * cos(th), mach * cs * sin(th), p, a.gamma, ub);
  } else if (a.ic_kind == IPM_IC_SHEAR) {
    // ghosts repeat the periodic interior
    const int iw = ii == 0 ? nx : (ii == nx + 1 ? 1 : ii);
    const int jw = jj == 0 ? ny : (jj == ny + 1 ? 1 : jj);
    const double ylo = a.y_lo + (jw - 1) * a.dy, yhi = ylo + a.dy;
    const double xc = a.x_lo + (iw - 0.5) * a.dx;
    const double amp = affine3(a.param[0], a.dparam[0], xi, P);
    const double ph = affine3(a.param[1], a.dparam[1], xi, P);
    const double hw = affine3(a.param[2], a.dparam[2], xi, P);
    const double ym = a.y_lo + 0.5 * a.dy * ny;
    const double f = fmax(fmin(yhi, ym + hw) - fmax(ylo, ym - hw), 0.0) / a.dy;
    const double v2 = amp * sin(a.param[3] * (xc + ph));
    const double rin = a.left[0], vin = a.left[1], rout = a.right[0], vout = a.right[1], p = a.left[3];
    const double rho = f * rin + (1.0 - f) * rout;
    ub[0] = rho;
    ub[1] = f * rin * vin + (1.0 - f) * rout * vout;
    ub[2] = rho * v2;
    ub[3] = p / (a.gamma - 1.0) + 0.5 * f * rin * (vin * vin + v2 * v2) + 0.5 * (1.0 - f) * rout * (vout * vout + v2 * v2);
  } else {
    // x-Riemann: exact cell average in x of the two states
    double pl[4], pr[4], UL[4], UR[4];
    for (int v = 0; v < 4; ++v) {
      pl[v] = affine3(a.left[v], a.dleft[v], xi, P);
      pr[v] = affine3(a.right[v], a.dright[v], xi, P);
    }
    prim4_to_cons(pl[0], pl[1], pl[2], pl[3], a.gamma, UL);
    prim4_to_cons(pr[0], pr[1], pr[2], pr[3], a.gamma, UR);
    const double x_left = a.x_lo + (ii - 1) * a.dx;
    const double x0 = affine3(a.x0, a.dx0, xi, P);
    const double frac = fmin(fmax((x0 - x_left) / a.dx, 0.0), 1.0);
#pragma unroll
    for (int k = 0; k < 4; ++k) ub[k] = frac * UL[k] + (1.0 - frac) * UR[k];
  }
}
#endif

}  // namespace ipm
