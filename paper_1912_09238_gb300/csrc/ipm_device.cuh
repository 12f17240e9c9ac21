// ipm_device.cuh -- device-side closures, fluxes and launch-argument structs of the IPM library.
//
// Entropy closures (Sec. 3.1: u_s = (grad s)^-1; Sec. 2, Eq. dualProblem: s_*; App. B for Euler):
//   per quadrature node the kernels need u_s(Lambda), its Jacobian grad u_s(Lambda) (symmetric,
//   stored packed a <= b) and s_*(Lambda) for the dual cost L of Eq. L.
//
// Euler (App. B, written with beta = -Lambda_E > 0 and k = 1/(gamma-1)):
//   ln rho = k (Lambda_1 - gamma - ln beta + |Lambda_v|^2 / (2 beta)),   v = Lambda_v / beta,
//   E = rho (1/beta + |v|^2/2),   s_* = (gamma-1) rho,   speed = max_d |v_d| + sqrt(gamma (gamma-1) / beta).
//   This is App. B's alpha with the exponent's gamma term taken as +2 gamma Lambda_E (the printed sign
//   does not invert grad s). Since grad s_* = u_s and grad rho = k u, the Jacobian is
//   grad u_s = rho [k g g^T + G],  g = (1, v, E/rho),
//   G = [[0, 0, 0], [0, I/beta, v/beta], [0, v^T/beta, 1/beta^2 + |v|^2/beta]].
// Bounded barrier (scalar): u = u_- + D sigma(Lambda), D = u_+ - u_-, grad u_s = D sigma (1 - sigma),
//   s_* = D softplus(Lambda) + u_- Lambda - D ln D.
// Quadratic: u = Lambda, grad u_s = I, s_* = |Lambda|^2 / 2 (stochastic Galerkin).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/ipm.h"

namespace ipm {

enum EntKind { ENT_QUADRATIC = 0, ENT_BARRIER = 1, ENT_EULER = 2 };
enum PhysKind { PHYS_BURGERS = 0, PHYS_EULER1D = 1, PHYS_EULER2D = 2 };

// per-cell status codes (values of ipm_status)
enum CellStatus {
  ST_OK = 0, ST_NOCONV = 3, ST_NOTSPD = 4, ST_INFEASIBLE = 5, ST_LINESEARCH = 6, ST_NONFINITE = 7, ST_TIMEOUT = 10
};

struct EntParams {
  double u_minus, u_plus, gamma;
};

__host__ __device__ constexpr int packed_count(int m) { return m * (m + 1) / 2; }
// entries of the packed lower triangle of the (NM+1) x (NM+1) matrix [[H, .], [g^T, .]] that the
// Newton kernel factorises (the extra row carries the gradient through the forward substitution)
__host__ __device__ constexpr size_t packed_aug_count(int NM) { return (size_t)(NM + 1) * (NM + 2) / 2; }
// index of (a, b), a <= b, in the packed upper triangle of an m x m symmetric matrix
__host__ __device__ constexpr int packed_ab(int a, int b, int m) { return a * m - a * (a - 1) / 2 + (b - a); }

#ifdef __CUDACC__
// ------------------------------------------------------------------------------------------------
// Closures: evaluate at one node. Lam[M] in; u[M], J[packed], sstar, speed out. Returns feasibility.
// ------------------------------------------------------------------------------------------------
template <int ENT, int M>
struct Closure;

template <int M>
struct Closure<ENT_QUADRATIC, M> {
  template <bool WANT_J>
  __device__ static bool eval(const double* L, const EntParams&, double* u, double* J, double& sstar) {
    double s = 0.0;
    bool ok = true;
#pragma unroll
    for (int a = 0; a < M; ++a) {
      u[a] = L[a];
      s = fma(L[a], L[a], s);
      ok = ok && isfinite(L[a]);
    }
    sstar = 0.5 * s;
    if (WANT_J) {
#pragma unroll
      for (int a = 0; a < M; ++a)
#pragma unroll
        for (int b = a; b < M; ++b) J[packed_ab(a, b, M)] = (a == b) ? 1.0 : 0.0;
    }
    return ok;
  }
  __device__ static bool feasible_sstar(const double* L, const EntParams& p, double& sstar) {
    double u[M];
    return eval<false>(L, p, u, nullptr, sstar);
  }
};

template <>
struct Closure<ENT_BARRIER, 1> {
  template <bool WANT_J>
  __device__ static bool eval(const double* L, const EntParams& p, double* u, double* J, double& sstar) {
    const double x = L[0];
    const double D = p.u_plus - p.u_minus;
    const double ex = exp(-fabs(x));
    const double inv = 1.0 / (1.0 + ex);
    const double sig = (x >= 0.0) ? inv : ex * inv;          // logistic(x) without overflow
    u[0] = p.u_minus + D * sig;
    if (WANT_J) J[0] = D * ex * inv * inv;                     // D sigma (1 - sigma)
    sstar = D * (fmax(x, 0.0) + log1p(ex)) + p.u_minus * x - D * log(D);
    return isfinite(x);
  }
  __device__ static bool feasible_sstar(const double* L, const EntParams& p, double& sstar) {
    double u[1];
    return eval<false>(L, p, u, nullptr, sstar);
  }
};

template <int M>
struct Closure<ENT_EULER, M> {
  static constexpr int D = M - 2;
  template <bool WANT_J>
  __device__ static bool eval(const double* L, const EntParams& p, double* u, double* J, double& sstar) {
    const double g = p.gamma;
    const double k = 1.0 / (g - 1.0);
    const double LE = L[M - 1];
    if (!(LE < 0.0)) {
      sstar = 0.0;
#pragma unroll
      for (int a = 0; a < M; ++a) u[a] = 0.0;
      return false;
    }
    const double beta = -LE;
    const double ib = 1.0 / beta;
    double lvsq = 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d) lvsq = fma(L[1 + d], L[1 + d], lvsq);
    const double lnrho = k * (L[0] - g - log(beta) + 0.5 * lvsq * ib);
    const double rho = exp(lnrho);
    double v[D > 0 ? D : 1];
    double vsq = 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      v[d] = L[1 + d] * ib;
      vsq = fma(v[d], v[d], vsq);
    }
    const double e = ib + 0.5 * vsq;                          // E / rho
    u[0] = rho;
#pragma unroll
    for (int d = 0; d < D; ++d) u[1 + d] = rho * v[d];
    u[M - 1] = rho * e;
    sstar = (g - 1.0) * rho;
    const bool ok = (rho > 0.0) && isfinite(rho) && isfinite(e);
    if (WANT_J) {
      double gv[M];
      gv[0] = 1.0;
#pragma unroll
      for (int d = 0; d < D; ++d) gv[1 + d] = v[d];
      gv[M - 1] = e;
#pragma unroll
      for (int a = 0; a < M; ++a)
#pragma unroll
        for (int b = a; b < M; ++b) {
          double G = 0.0;
          if (a >= 1 && a <= D && b >= 1 && b <= D) G = (a == b) ? ib : 0.0;
          else if (a >= 1 && a <= D && b == M - 1) G = v[a - 1] * ib;
          else if (a == M - 1 && b == M - 1) G = ib * ib + vsq * ib;
          J[packed_ab(a, b, M)] = rho * fma(k * gv[a], gv[b], G);
        }
    }
    return ok;
  }
  __device__ static bool feasible_sstar(const double* L, const EntParams& p, double& sstar) {
    double u[M];
    return eval<false>(L, p, u, nullptr, sstar);
  }
  // fastest signal speed from the dual state (used at the converged duals)
  __device__ static double speed_from_dual(const double* L, const EntParams& p) {
    const double beta = -L[M - 1];
    double vmax = 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d) vmax = fmax(vmax, fabs(L[1 + d] / beta));
    return vmax + sqrt(p.gamma * (p.gamma - 1.0) / beta);
  }
};

// grad s(u): entropy variables of a conserved state (initial duals only).
template <int ENT, int M>
__device__ inline void entropy_gradient(const double* u, const EntParams& p, double* out) {
  if (ENT == ENT_QUADRATIC) {
#pragma unroll
    for (int a = 0; a < M; ++a) out[a] = u[a];
  } else if (ENT == ENT_BARRIER) {
    out[0] = log(u[0] - p.u_minus) - log(p.u_plus - u[0]);
  } else {
    constexpr int D = M - 2;
    const double rho = u[0], E = u[M - 1];
    double msq = 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d) msq = fma(u[1 + d], u[1 + d], msq);
    const double eps = E - 0.5 * msq / rho;                   // internal energy density
    out[0] = -log(pow(rho, -p.gamma) * eps) - 0.5 * msq / (rho * eps) + p.gamma;
#pragma unroll
    for (int d = 0; d < D; ++d) out[1 + d] = u[1 + d] / eps;
    out[M - 1] = -rho / eps;
  }
}

// ------------------------------------------------------------------------------------------------
// Physics on conserved states (Burgers App. A; Euler Sec. 7.1).
// ------------------------------------------------------------------------------------------------
template <int PHYS, int M>
struct Physics;

template <>
struct Physics<PHYS_BURGERS, 1> {
  __device__ static void flux(const double* u, double, double* f) { f[0] = 0.5 * u[0] * u[0]; }
  __device__ static double speed(const double* u, double) { return fabs(u[0]); }
};

template <>
struct Physics<PHYS_EULER1D, 3> {
  __device__ static void flux(const double* u, double g, double* f) {
    const double v = u[1] / u[0];
    const double p = (g - 1.0) * (u[2] - 0.5 * u[1] * v);
    f[0] = u[1];
    f[1] = u[1] * v + p;
    f[2] = (u[2] + p) * v;
  }
  __device__ static double speed(const double* u, double g) {
    const double v = u[1] / u[0];
    const double p = (g - 1.0) * (u[2] - 0.5 * u[1] * v);
    return fabs(v) + sqrt(g * p / u[0]);
  }
};

#endif  // __CUDACC__

// ------------------------------------------------------------------------------------------------
// Launch arguments
// ------------------------------------------------------------------------------------------------
struct Tables {
  const double* Phi;     // [Q][N]  phi_i(xi_k)
  const double* PhiT;    // [N][Q]
  const double* w;       // [Q]     weights with the density folded in
  const double* nodes;   // [Q][p]
  const uint32_t* pairs; // [N(N+1)/2] (i << 16) | j with i >= j, row-major over i
  int N, Q, p;
};

struct StepScalars {
  unsigned long long smax_bits;  // max signal speed over cells and nodes (positive double bits)
  unsigned long long fixed_smax_bits; // speed of the fixed (Dirichlet) ghosts
  int work_counter;              // persistent-queue counter of the Newton kernel
  int update_counter;
  int n_cta_items;               // split queue: items for the CTA-per-cell kernel (the rest: one warp per cell)
  int warp_counter;              // split queue: counter of the warp-per-cell kernel
  double t;                      // current time
  double dt;                     // last time step
  double residual;               // last steady residual
  int64_t steps;
  int64_t newton_iters;
  int max_iters;
  int failed_cells;
  int first_failed_cell;
  int first_status;
  int tc_timeouts;               // bounded tensor-core / bulk-copy waits that ran out (mixed path)
  int level_cap;                 // adaptive meshes: highest level the update may assign (Algorithm 4 stages)
  unsigned long long factorizations;       // Cholesky factorisations since the last reduction
  unsigned long long last_factorizations;  // ... of the last solve (frozen-Hessian statistics)
  int fp32_fallbacks;                      // FP32-factor mode: factorisations redone in FP64 (cumulative)
  unsigned long long cached_checks;        // cells whose convergence check came from their moment image
  unsigned long long last_cached_checks;   // ... of the last solve
  int tc_stuck;                  // sticky: a CTA could not drain its tensor-core work after a timeout
  unsigned long long hessian_ns;        // mixed path: tensor-core Hessian phases since the last reduction (ns, summed over CTAs)
  unsigned long long hessian_count;     // ... and how many
  unsigned long long last_hessian_ns;   // ... of the last solve
  unsigned long long last_hessian_count;
};

// Mixed-precision Hessian (tensor cores): tiling of H_ab = Phi^T diag(w J_ab) Phi as MMAs with
// rows (ab, i) of the per-cell operand, columns j, and the quadrature nodes as the K dimension.
struct MixedTiles {
  const uint8_t* phi_img;  // [chunk][hi, lo][n_pad x kc] BF16 K-major images of Phi (B operand)
  const float* phiT32;     // [N][Q] Phi^T in FP32 (builds the A operand)
  const float* phi32c;     // [chunk][n_rows][kcp] the same by K-chunk, rows padded to kcp (bulk-copy source)
  int n_rows;              // rows of phi32c (the table's N)
  int kcp;                 // kc + 4: row stride of phi32c (shifts consecutive rows by four banks)
  uint32_t off_ph;         // shared-memory offset of two staged phi32c chunks, 0: no staging
  int n_pad;               // N rounded up to a multiple of 16 (MMA N)
  int kc;                  // nodes per K-chunk (multiple of 16)
  int chunks;              // ceil(Q / kc)
  int tiles;               // ceil(B N / 128) row tiles of 128 (MMA M)
  int tpp;                 // row tiles per pass (accumulators resident in tensor memory at once)
  int tmem_cols;           // allocated tensor-memory columns (power of two >= 32)
  int abuf;                // A staging buffers (2: the next chunk is built while the MMAs of this one run)
  int stack;               // 1: B = [B_hi; B_lo] as one operand, two accumulators of n_pad columns per row tile
};

struct NewtonArgs {
  Tables tab;
  EntParams ent;
  double* uhat;          // [C][N][m]
  double* lam;           // [C][N][m]
  double* unode;         // [C][m][Q]  nodal states at the final duals
  int* iters;            // [C]
  int* status;           // [C]
  double* hwork;         // global workspace for packed Hessians when they do not fit in shared memory
  size_t hwork_stride;   // doubles per CTA slot
  StepScalars* sc;
  const int* cell_list;  // explicit cell indices, or nullptr for the interior of the mesh
  int n_work;            // number of cells to process
  int nx, gy;            // interior mapping: cell = (w / nx + gy) * (nx + 2) + (w % nx + 1)
  int one_step;          // 1: exactly one damped Newton step (Algorithm 2)
  double tau, armijo_c, slack_rel;
  int max_newton, max_halvings;
  int track_speed;       // 1: fold the nodal signal speeds of the result into sc->smax_bits
  double* h_dump;        // non-null: assemble the Hessian at the current duals, store it packed
                         // [work item][NM(NM+1)/2] and stop (no Newton update)
  int hessian_reuse;     // 0: Newton; 1: reuse the factor within a solve; 2: also across solves
  double reuse_ratio;    // reuse while the residual falls at least by this factor per full step
  double* factor_store;  // hessian_reuse 2: [cell][NM(NM+1)/2 + NM] kept factor and reciprocal pivots
  size_t factor_stride;
  int* factor_valid;     // [cell]
  const int* level;      // adaptive meshes: refinement level per cell (nullptr: every cell at tab.N)
  int lev_n[8];          // moments per level (graded prefixes of the table's basis)
  // quadrature per level (nested Clenshaw-Curtis rules): nodes of each level's rule (a prefix of the
  // table's nodes) and its weights [level][tab.Q]; lev_w == nullptr: every level uses tab.w over tab.Q
  int lev_q[8];
  const double* lev_w;
  const int* level_next; // adaptive meshes: the level each cell takes in this step's update (wave speeds
                         // are taken at that level's nodes), or nullptr
  const int* q_eval;     // per-level rules: nodes at which each cell's nodal states are written (the
                         // largest new level's rule over its stencil); the rest of its row is zeroed
  // split queue of adaptive meshes (k_order groups the cells by kernel): the items are
  // cell_list[*first_dev .. *count_dev) taken through the counter *queue; nullptr: 0, n_work and
  // sc->work_counter
  int* queue;
  const int* first_dev;
  const int* count_dev;
  // moment images (nullptr: off): img[cell] holds S = sum_k w_k u(Lambda(xi_k)) phi(xi_k) of the duals
  // img_lam[cell] that the cell's last successful solve ended at, img_smax[cell] the wave speed at those
  // duals' nodal states; img_valid[cell] = level + 1 when the three belong together (0: none)
  double* img;           // [cell][NM]
  double* img_lam;       // [cell][NM]
  double* img_smax;      // [cell]
  int* img_valid;        // [cell]
  // 1-D Lax-Friedrichs update folded into the Newton launch (nullptr: off). With nu = dx / (2 dt) the
  // update of cell j is u_hat_j = A_j - (dt/dx) B_j with A_j = P(w (u_l + u_r) / 2) and
  // B_j = P(w (f(u_r) - f(u_l)) / 2) over the nodal states of its two neighbours, neither of which
  // needs dt; the CTA that finishes the last neighbour of j forms lf_a[j] = A_j and lf_b[j] = B_j.
  // lf_cnt[j] counts the finished neighbours (zeroed before the launch).
  double* lf_a;          // [cell][NM]
  double* lf_b;          // [cell][NM]
  int* lf_cnt;           // [cell]
  int bc_left, bc_right;
  MixedTiles mx;         // mixed path only
  uint32_t off_h, off_a, off_b;  // shared-memory byte offsets: packed H, A staging, Phi chunks
  // split factorisation (tensor-core trailing updates): shared-memory offset of the digit slices and
  // row exponents, rows per slice, tensor-memory accumulator sets (1 or 2)
  uint32_t off_s;
  int s_rows, s_nbuf;
  double* f_dump;        // non-null: factorise the augmented Hessian at the current duals, store L packed
                         // [work item][NM(NM+1)/2] and stop (no Newton update)
};

struct Update1DArgs {
  Tables tab;
  double* uhat;          // [C][N][m]  (written for interior cells and outflow/periodic ghosts)
  double* lam;           // [C][N][m]  (ghost copies only)
  const double* unode;   // [C][m][Q]
  double* cell_resid;    // [C] per-cell contribution to the steady residual
  StepScalars* sc;
  int nx;
  int bc_left, bc_right;
  double dx, cfl, t_end, gamma;
  double dt_override;    // > 0: use this dt instead of the CFL rule
};

// 2-D structured mesh on the device: cell areas [ny][nx]; x-faces [ny][nx+1] and y-faces [ny+1][nx]
// as (n_x, n_y, length) with the unit normal pointing to increasing i (x-faces) or j (y-faces).
struct Mesh2DDev {
  const double* area;
  const double* xf;
  const double* yf;
  int nx, ny;
  double h_min;          // min over cells of area / longest face
};

struct Update2DArgs {
  Tables tab;
  Mesh2DDev mesh;
  double* uhat;          // [(ny+2)(nx+2)][N][m]
  const double* unode;   // [(ny+2)(nx+2)][m][Q]
  double* cell_resid;    // [(ny+2)(nx+2)] area-weighted |change of the density mean|
  StepScalars* sc;
  int bc[4];             // left, right, bottom, top (ipm_bc)
  double cfl, t_end, gamma;
  double dt_override;    // > 0: use this dt
  int clip;              // 1: clip the step to t_end
  // adaptive meshes (Algorithm 3): level per cell, or nullptr
  int* level;
  double* lam;           // [(ny+2)(nx+2)][N][m]  duals (truncated to the new level)
  int n_levels;
  int lev_n[8], lev_prev[8];   // moments of each level and of the level's lower-degree part
  double delta_lo, delta_hi;
  int* level_next;       // the new level of every cell, set before the Newton kernel (k_next_levels)
  int* q_eval;           // per-level rules: nodes each cell's nodal states must cover (k_eval_q)
  int lev_q[8];          // nodes of each level's rule (tab.Q for all with one shared rule)
  const double* lev_w;   // per-level rules: weights [level][tab.Q], or nullptr
};

#ifdef __CUDACC__
// positive doubles order like their bit patterns
__device__ inline void atomic_max_pos(unsigned long long* addr, double v) {
  if (v > 0.0) atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

// fastest signal speed of a nodal state: |u| (Burgers), max_d |v_d| + c (Euler)
template <int PHYS, int M>
__device__ __forceinline__ double node_speed(const double* u, double gamma);

template <>
__device__ __forceinline__ double node_speed<PHYS_BURGERS, 1>(const double* u, double) { return fabs(u[0]); }
template <>
__device__ __forceinline__ double node_speed<PHYS_EULER1D, 3>(const double* u, double g) {
  const double v = u[1] / u[0];
  const double p = (g - 1.0) * (u[2] - 0.5 * u[1] * v);
  return fabs(v) + sqrt(g * p / u[0]);
}
template <>
__device__ __forceinline__ double node_speed<PHYS_EULER2D, 4>(const double* u, double g) {
  const double v1 = u[1] / u[0], v2 = u[2] / u[0];
  const double p = (g - 1.0) * (u[3] - 0.5 * (u[1] * v1 + u[2] * v2));
  return fmax(fabs(v1), fabs(v2)) + sqrt(g * p / u[0]);
}

// cell index of the left (side < 0) or right neighbour of interior cell j of a 1-D mesh, resolved
// through the boundary condition: outflow reads the cell itself, periodic the opposite end,
// Dirichlet the fixed ghost
__device__ __forceinline__ int neighbour(int j, int nx, int side, int bc) {
  // side -1: left neighbour of j, +1: right neighbour
  if (side < 0) {
    if (j > 1) return j - 1;
    return bc == IPM_BC_OUTFLOW ? 1 : (bc == IPM_BC_PERIODIC ? nx : 0);
  }
  if (j < nx) return j + 1;
  return bc == IPM_BC_OUTFLOW ? nx : (bc == IPM_BC_PERIODIC ? 1 : nx + 1);
}

// physical flux of the 1-D systems (App. A Burgers; Sec. 7.1 Euler)
template <int PHYS, int M>
struct Flux1D;
template <>
struct Flux1D<PHYS_BURGERS, 1> {
  __device__ static void f(const double* u, double, double* out) { out[0] = 0.5 * u[0] * u[0]; }
};
template <>
struct Flux1D<PHYS_EULER1D, 3> {
  __device__ static void f(const double* u, double g, double* out) {
    const double v = u[1] / u[0];
    const double p = (g - 1.0) * (u[2] - 0.5 * u[1] * v);
    out[0] = u[1];
    out[1] = fma(u[1], v, p);
    out[2] = (u[2] + p) * v;
  }
};

// F(u).n and |v.n| + c for the 2-D Euler system
__device__ __forceinline__ double euler2d_normal_flux(const double* u, double nx, double ny, double g, double* f) {
  const double rho = u[0], ir = 1.0 / rho;
  const double v1 = u[1] * ir, v2 = u[2] * ir;
  const double p = (g - 1.0) * (u[3] - 0.5 * (u[1] * v1 + u[2] * v2));
  const double vn = v1 * nx + v2 * ny;
  f[0] = rho * vn;
  f[1] = fma(u[1], vn, p * nx);
  f[2] = fma(u[2], vn, p * ny);
  f[3] = (u[3] + p) * vn;
  return fabs(vn) + sqrt(g * p * ir);
}

// Rusanov flux from a (behind) to b (ahead) across unit normal n
__device__ __forceinline__ void rusanov2d(const double* ua, const double* ub, double nx, double ny, double g,
                                          double* out) {
  double fa[4], fb[4];
  const double sa = euler2d_normal_flux(ua, nx, ny, g, fa);
  const double sb = euler2d_normal_flux(ub, nx, ny, g, fb);
  const double s = fmax(sa, sb);
#pragma unroll
  for (int c = 0; c < 4; ++c) out[c] = 0.5 * (fa[c] + fb[c]) - 0.5 * s * (ub[c] - ua[c]);
}

__device__ __forceinline__ void reflect(const double* u, double nx, double ny, double* out) {
  const double mn = u[1] * nx + u[2] * ny;
  out[0] = u[0];
  out[1] = u[1] - 2.0 * mn * nx;
  out[2] = u[2] - 2.0 * mn * ny;
  out[3] = u[3];
}

__device__ __forceinline__ int cell2d(int i, int j, int nx) { return (j + 1) * (nx + 2) + (i + 1); }

// state beyond a boundary face: the neighbour cell index, or -1 for the cell itself (outflow),
// or -2 for the reflected state (slip wall)
__device__ __forceinline__ int outside(int bc, int wrap_cell, int ghost_cell) {
  if (bc == IPM_BC_PERIODIC) return wrap_cell;
  if (bc == IPM_BC_DIRICHLET) return ghost_cell;
  if (bc == IPM_BC_SLIP_WALL) return -2;
  return -1;
}

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
#endif  // __CUDACC__

}  // namespace ipm
