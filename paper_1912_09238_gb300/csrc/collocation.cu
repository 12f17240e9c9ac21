// collocation.cu -- Stochastic Collocation (SC), the non-intrusive baseline the paper compares IPM
// with (Sec. 2, the collocation paragraph; Sec. 7, the IPM-versus-SC comparisons), on the same meshes
// and with the same numerical flux as the IPM moment update.
//
// Every quadrature node xi_k runs the deterministic finite-volume scheme on its own nodal state
// u_k(x, t) = u(x, t, xi_k), starting from the exact nodal cell averages of the initial data, with its
// own time step dt_k = CFL h / s_max,k (s_max,k over the interior cells and the Dirichlet ghosts at
// node k; in 1-D the Lax-Friedrichs viscosity dx / (2 dt_k) of the node's own step), until t_k
// reaches t_end (the last step clipped) or, for steady problems (t_end = 0), until its residual
// sum_c A_c |rho_c^{n+1} - rho_c^n| (A_c = dx in 1-D) falls below the tolerance. The moments are
// u_hat_i = sum_k w_k u_k phi_i(xi_k). The nodes advance in lockstep on the device (a finished node
// is copied through), which gives the same per-node result as independent runs.
//
// Layout: nodal states [cell][variable][node] over the ghost-inclusive cells, two buffers.
// k_sc_step: lane = node inside a tile of 32 nodes (coalesced loads across the lanes), warp = a run
//   of ch consecutive interior cells (along x), whose shared x-face fluxes are computed once; ch is
//   the longest run (8, 4, 2 or 1) that still gives 8 warps per SM (the step is FP64-bound: shorter
//   runs recompute fluxes and measured slower on the 2000-cell Sod tube);
//   per block and node the largest wave speed of the new states and the residual sum, reduced over
//   the warps in a fixed order into part_*[block][node].
// k_sc_nodes: one block; per node: fold the partials in block order, advance t_k and the step count,
//   set the next dt_k (0 once the node has finished) and count the running nodes.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ic.cuh"
#include "ipm_host.h"

namespace ipm {

constexpr int SC_W = 8;        // warps per block
constexpr int SC_T = 32 * SC_W;
constexpr int SC_GRAPH_STEPS = 16;   // steps per captured graph (even: the buffers swap back)

struct ScStepArgs {
  int nx, ny, Q, n_interior;
  int ch;                     // consecutive interior cells per warp
  int bc[4];
  double dx, gamma;
  Mesh2DDev mesh;
  const double* u_in;         // [cell][m][Q]
  double* u_out;
  const double* node_dt;      // [Q]: this step's dt of every node, 0 = finished
  double* part_smax;          // [gridDim.x][Q]
  double* part_res;
  int update;                 // 0: only the speed partials of u_in (initial time step)
};

template <int PHYS, int M>
__device__ __forceinline__ void sc_load(const double* u, int cell, int Q, int q, double* v) {
  const double* p = u + (size_t)cell * M * Q + q;
#pragma unroll
  for (int k = 0; k < M; ++k) v[k] = p[(size_t)k * Q];
}

template <int M>
__device__ __forceinline__ void sc_store(double* u, int cell, int Q, int q, const double* v) {
  double* p = u + (size_t)cell * M * Q + q;
#pragma unroll
  for (int k = 0; k < M; ++k) p[(size_t)k * Q] = v[k];
}

// 1-D: cells j0..j1 (ghost-inclusive indices, 1 <= j0 <= j1 <= nx) of node q
template <int PHYS, int M>
__device__ __forceinline__ void sc_run1d(const ScStepArgs& a, int q, double dt, int j0, int j1, double& smax,
                                         double& res) {
  const int nx = a.nx, Q = a.Q;
  double uc[M], un[M];
  if (!a.update || dt == 0.0) {
    for (int j = j0; j <= j1; ++j) {
      sc_load<PHYS, M>(a.u_in, j, Q, q, uc);
      smax = fmax(smax, node_speed<PHYS, M>(uc, a.gamma));
      if (a.update) sc_store<M>(a.u_out, j, Q, q, uc);
    }
    if (a.update && j0 == 1) {
      sc_load<PHYS, M>(a.u_in, 0, Q, q, uc);
      sc_store<M>(a.u_out, 0, Q, q, uc);
    }
    if (a.update && j1 == nx) {
      sc_load<PHYS, M>(a.u_in, nx + 1, Q, q, uc);
      sc_store<M>(a.u_out, nx + 1, Q, q, uc);
    }
    return;
  }
  const double nu = a.dx / (2.0 * dt), r = dt / a.dx;
  double fc[M], fn[M], gl[M], gr[M];
  sc_load<PHYS, M>(a.u_in, neighbour(j0, nx, -1, a.bc[0]), Q, q, un);
  sc_load<PHYS, M>(a.u_in, j0, Q, q, uc);
  Flux1D<PHYS, M>::f(un, a.gamma, fn);
  Flux1D<PHYS, M>::f(uc, a.gamma, fc);
#pragma unroll
  for (int k = 0; k < M; ++k) gl[k] = 0.5 * (fn[k] + fc[k]) - nu * (uc[k] - un[k]);
  for (int j = j0; j <= j1; ++j) {
    sc_load<PHYS, M>(a.u_in, neighbour(j, nx, 1, a.bc[1]), Q, q, un);
    Flux1D<PHYS, M>::f(un, a.gamma, fn);
    double nw[M];
#pragma unroll
    for (int k = 0; k < M; ++k) {
      gr[k] = 0.5 * (fc[k] + fn[k]) - nu * (un[k] - uc[k]);
      nw[k] = uc[k] - r * (gr[k] - gl[k]);
    }
    sc_store<M>(a.u_out, j, Q, q, nw);
    res += a.dx * fabs(nw[0] - uc[0]);
    smax = fmax(smax, node_speed<PHYS, M>(nw, a.gamma));
    // ghost copies of outflow and periodic ends (Dirichlet ghosts keep their state in both buffers)
    if (j == 1 && a.bc[0] == IPM_BC_OUTFLOW) sc_store<M>(a.u_out, 0, Q, q, nw);
    if (j == 1 && a.bc[1] == IPM_BC_PERIODIC) sc_store<M>(a.u_out, nx + 1, Q, q, nw);
    if (j == nx && a.bc[1] == IPM_BC_OUTFLOW) sc_store<M>(a.u_out, nx + 1, Q, q, nw);
    if (j == nx && a.bc[0] == IPM_BC_PERIODIC) sc_store<M>(a.u_out, 0, Q, q, nw);
#pragma unroll
    for (int k = 0; k < M; ++k) {
      uc[k] = un[k];
      fc[k] = fn[k];
      gl[k] = gr[k];
    }
  }
}

// 2-D: flattened interior cells c0..c1 (row-major, c = j nx + i) of node q
__device__ __forceinline__ void sc_face_state(const ScStepArgs& a, int o, const double* uc, double nx_, double ny_,
                                              int q, double* un) {
  if (o >= 0) {
    sc_load<PHYS_EULER2D, 4>(a.u_in, o, a.Q, q, un);
  } else if (o == -1) {
#pragma unroll
    for (int k = 0; k < 4; ++k) un[k] = uc[k];
  } else {
    reflect(uc, nx_, ny_, un);
  }
}

__device__ __forceinline__ void sc_run2d(const ScStepArgs& a, int q, double dt, int c0, int c1, double& smax,
                                         double& res) {
  const int nx = a.nx, ny = a.ny, Q = a.Q;
  const double g = a.gamma;
  double uc[4], un[4], gxl[4], f[4];
  if (!a.update || dt == 0.0) {
    for (int c = c0; c <= c1; ++c) {
      const int cell = cell2d(c % nx, c / nx, nx);
      sc_load<PHYS_EULER2D, 4>(a.u_in, cell, Q, q, uc);
      smax = fmax(smax, node_speed<PHYS_EULER2D, 4>(uc, g));
      if (a.update) sc_store<4>(a.u_out, cell, Q, q, uc);
    }
    return;
  }
  bool have_left = false;
  for (int c = c0; c <= c1; ++c) {
    const int i = c % nx, j = c / nx;
    const int cell = cell2d(i, j, nx);
    sc_load<PHYS_EULER2D, 4>(a.u_in, cell, Q, q, uc);
    const double* xl = a.mesh.xf + ((size_t)j * (nx + 1) + i) * 3;
    const double* xr = xl + 3;
    const double* yb = a.mesh.yf + ((size_t)j * nx + i) * 3;
    const double* yt = a.mesh.yf + ((size_t)(j + 1) * nx + i) * 3;
    if (!have_left || i == 0) {
      const int nl = i > 0 ? cell2d(i - 1, j, nx) : outside(a.bc[0], cell2d(nx - 1, j, nx), cell2d(-1, j, nx));
      sc_face_state(a, nl, uc, xl[0], xl[1], q, un);
      rusanov2d(un, uc, xl[0], xl[1], g, f);
#pragma unroll
      for (int k = 0; k < 4; ++k) gxl[k] = xl[2] * f[k];
    }
    double acc[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] = -gxl[k];
    const int nr = i < nx - 1 ? cell2d(i + 1, j, nx) : outside(a.bc[1], cell2d(0, j, nx), cell2d(nx, j, nx));
    sc_face_state(a, nr, uc, xr[0], xr[1], q, un);
    rusanov2d(uc, un, xr[0], xr[1], g, f);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      gxl[k] = xr[2] * f[k];             // the right face of this cell is the left face of the next
      acc[k] += gxl[k];
    }
    have_left = true;
    const int nb = j > 0 ? cell2d(i, j - 1, nx) : outside(a.bc[2], cell2d(i, ny - 1, nx), cell2d(i, -1, nx));
    sc_face_state(a, nb, uc, yb[0], yb[1], q, un);
    rusanov2d(un, uc, yb[0], yb[1], g, f);
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] = fma(-yb[2], f[k], acc[k]);
    const int nt = j < ny - 1 ? cell2d(i, j + 1, nx) : outside(a.bc[3], cell2d(i, 0, nx), cell2d(i, ny, nx));
    sc_face_state(a, nt, uc, yt[0], yt[1], q, un);
    rusanov2d(uc, un, yt[0], yt[1], g, f);
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] = fma(yt[2], f[k], acc[k]);
    const double area = a.mesh.area[(size_t)j * nx + i];
    const double r = dt / area;
    double nw[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) nw[k] = fma(-r, acc[k], uc[k]);
    sc_store<4>(a.u_out, cell, Q, q, nw);
    res += area * fabs(nw[0] - uc[0]);
    smax = fmax(smax, node_speed<PHYS_EULER2D, 4>(nw, g));
  }
}

template <int PHYS, int M>
__global__ void __launch_bounds__(SC_T) k_sc_step(ScStepArgs a) {
  __shared__ double s_max[SC_W][32], s_res[SC_W][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int q = blockIdx.y * 32 + lane;
  const int c0 = (blockIdx.x * SC_W + warp) * a.ch;       // first flattened interior cell of the warp
  double smax = 0.0, res = 0.0;
  if (q < a.Q && c0 < a.n_interior) {
    const double dt = a.node_dt[q];
    const int c1 = min(c0 + a.ch, a.n_interior) - 1;
    if constexpr (PHYS == PHYS_EULER2D) sc_run2d(a, q, dt, c0, c1, smax, res);
    else sc_run1d<PHYS, M>(a, q, dt, c0 + 1, c1 + 1, smax, res);
  }
  s_max[warp][lane] = smax;
  s_res[warp][lane] = res;
  __syncthreads();
  if (warp == 0 && q < a.Q) {
    double mx = 0.0, rs = 0.0;
#pragma unroll
    for (int w = 0; w < SC_W; ++w) {
      mx = fmax(mx, s_max[w][lane]);
      rs += s_res[w][lane];
    }
    a.part_smax[(size_t)blockIdx.x * a.Q + q] = mx;
    a.part_res[(size_t)blockIdx.x * a.Q + q] = rs;
  }
}

struct ScNodeArgs {
  int Q, n_parts, init, steady;
  double h, cfl, t_end, tol;
  const double* part_smax;
  const double* part_res;
  const double* fixed_smax;   // [Q] wave speed of the Dirichlet ghosts (0 without them)
  double* t;
  long long* steps;
  double* res;
  double* dt;
  int* n_active;
};

__global__ void __launch_bounds__(256) k_sc_nodes(ScNodeArgs a) {
  __shared__ int s_cnt[256 / 32];
  int cnt = 0;
  for (int q = threadIdx.x; q < a.Q; q += blockDim.x) {
    if (a.init) {
      a.t[q] = 0.0;
      a.steps[q] = 0;
      a.res[q] = INFINITY;
    } else if (a.dt[q] > 0.0) {
      a.t[q] += a.dt[q];
      a.steps[q] += 1;
      double r = 0.0;
      for (int b = 0; b < a.n_parts; ++b) r += a.part_res[(size_t)b * a.Q + q];
      a.res[q] = r;
    }
    double smax = a.fixed_smax[q];
    for (int b = 0; b < a.n_parts; ++b) smax = fmax(smax, a.part_smax[(size_t)b * a.Q + q]);
    const double t = a.t[q];
    const bool active = a.steady ? !(a.res[q] < a.tol) : t < a.t_end;
    double d = 0.0;
    if (active) {
      d = a.cfl * a.h / smax;
      if (a.t_end > 0.0 && t + d > a.t_end) d = a.t_end - t;
    }
    a.dt[q] = d;
    cnt += active ? 1 : 0;
  }
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0) s_cnt[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int tot = 0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) tot += s_cnt[w];
    *a.n_active = tot;
  }
}

// initial nodal states: exact cell averages of the data at every node, in both buffers; 1-D outflow
// and periodic ghosts take the state of the cell they copy
struct ScInitArgs {
  IC1D ic1;
  IC2D ic2;
  const double* nodes;   // [Q][p]
  int p, Q, n_cells, nx, bc_left, bc_right;
  double* u0;
  double* u1;
};

template <int PHYS, int M>
__global__ void k_sc_init(ScInitArgs a) {
  const size_t total = (size_t)a.n_cells * a.Q;
  for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int cell = (int)(t / a.Q), q = (int)(t % a.Q);
    double xi[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < a.p; ++d) xi[d] = a.nodes[(size_t)q * a.p + d];
    double ub[M];
    if constexpr (PHYS == PHYS_EULER2D) {
      ic2d_average(a.ic2, cell % (a.nx + 2), cell / (a.nx + 2), xi, a.p, ub);
    } else {
      int src = cell;
      if (cell == 0) src = a.bc_left == IPM_BC_OUTFLOW ? 1 : (a.bc_left == IPM_BC_PERIODIC ? a.nx : 0);
      if (cell == a.nx + 1) src = a.bc_right == IPM_BC_OUTFLOW ? a.nx : (a.bc_right == IPM_BC_PERIODIC ? 1 : a.nx + 1);
      ic1d_average<M>(a.ic1, src, xi, a.p, ub);
    }
#pragma unroll
    for (int k = 0; k < M; ++k) {
      a.u0[((size_t)cell * M + k) * a.Q + q] = ub[k];
      a.u1[((size_t)cell * M + k) * a.Q + q] = ub[k];
    }
  }
}

// largest wave speed of the Dirichlet ghost cells, per node
template <int PHYS, int M>
__global__ void k_sc_fixed(const double* u, const int* ghosts, int n_ghosts, int Q, double gamma, double* out) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < Q; q += gridDim.x * blockDim.x) {
    double s = 0.0, v[M];
    for (int k = 0; k < n_ghosts; ++k) {
      sc_load<PHYS, M>(u, ghosts[k], Q, q, v);
      s = fmax(s, node_speed<PHYS, M>(v, gamma));
    }
    out[q] = s;
  }
}

// moments of every cell: u_hat[c][i][a] = sum_q w_q phi_i(xi_q) u[c][a][q]; one block per cell
template <int M>
__global__ void __launch_bounds__(256) k_sc_moments(const double* u, const double* PhiT, const double* w, int N, int Q,
                                                    int n_cells, double* uhat) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = blockIdx.x; c < n_cells; c += gridDim.x) {
    const double* uc = u + (size_t)c * M * Q;
    for (int i = warp; i < N; i += 8) {
      double s[M];
#pragma unroll
      for (int k = 0; k < M; ++k) s[k] = 0.0;
      for (int q = lane; q < Q; q += 32) {
        const double wp = w[q] * PhiT[(size_t)i * Q + q];
#pragma unroll
        for (int k = 0; k < M; ++k) s[k] = fma(wp, uc[(size_t)k * Q + q], s[k]);
      }
#pragma unroll
      for (int k = 0; k < M; ++k) {
        const double v = warp_sum(s[k]);
        if (lane == 0) uhat[((size_t)c * N + i) * M + k] = v;
      }
    }
  }
}

}  // namespace ipm

using namespace ipm;

struct ipm_sc {
  ipm_problem prob;
  HostTables tab;
  Mesh2DHost mesh;
  int m = 0, phys = 0, Q = 0, N = 0, n_cells = 0, n_interior = 0;
  bool is2d = false;
  double h = 0.0, tol = 0.0;
  int grid_x = 0, grid_y = 0, ch = 8;
  int cur = 0;                     // buffer holding the current states
  long long steps = 0;             // lockstep steps launched
  int active = 0;                  // running nodes after the last step (host copy)
  cudaStream_t stream = nullptr;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  cudaEvent_t ev[2] = {nullptr, nullptr};
  double *d_u[2] = {nullptr, nullptr};
  double *d_PhiT = nullptr, *d_w = nullptr, *d_nodes = nullptr, *d_area = nullptr, *d_xf = nullptr, *d_yf = nullptr;
  double *d_part_smax = nullptr, *d_part_res = nullptr, *d_fixed = nullptr, *d_t = nullptr, *d_res = nullptr,
         *d_dt = nullptr;
  long long* d_steps = nullptr;
  int* d_active = nullptr;
  int* d_ghosts = nullptr;
  int* h_active = nullptr;         // pinned
  std::string err;
};

static ipm_status sc_fail(ipm_sc* s, ipm_status st, const std::string& msg) {
  if (s) s->err = msg;
  else set_global_error(msg);
  return st;
}

#define SC_CK(s, call)                                                                                  \
  do {                                                                                                  \
    cudaError_t e_ = (call);                                                                            \
    if (e_ != cudaSuccess) {                                                                            \
      cudaGetLastError();                                                                               \
      return sc_fail(s, e_ == cudaErrorMemoryAllocation ? IPM_ENOMEM : IPM_ECUDA,                       \
                     std::string(#call) + ": " + cudaGetErrorString(e_));                              \
    }                                                                                                   \
  } while (0)

template <typename T>
static cudaError_t sc_upload(T** dst, const std::vector<T>& src) {
  cudaError_t e = cudaMalloc((void**)dst, std::max<size_t>(1, src.size()) * sizeof(T));
  if (e != cudaSuccess || src.empty()) return e;
  return cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

static ScStepArgs sc_step_args(const ipm_sc* s, int from, int update) {
  ScStepArgs a;
  a.nx = s->prob.nx;
  a.ny = s->is2d ? s->prob.ny : 1;
  a.Q = s->Q;
  a.n_interior = s->n_interior;
  a.ch = s->ch;
  a.bc[0] = s->prob.bc_left;
  a.bc[1] = s->prob.bc_right;
  a.bc[2] = s->prob.bc_bottom;
  a.bc[3] = s->prob.bc_top;
  a.dx = (s->prob.x_hi - s->prob.x_lo) / s->prob.nx;
  a.gamma = s->prob.gamma;
  a.mesh.area = s->d_area;
  a.mesh.xf = s->d_xf;
  a.mesh.yf = s->d_yf;
  a.mesh.nx = s->prob.nx;
  a.mesh.ny = a.ny;
  a.mesh.h_min = s->h;
  a.u_in = s->d_u[from];
  a.u_out = s->d_u[from ^ 1];
  a.node_dt = s->d_dt;
  a.part_smax = s->d_part_smax;
  a.part_res = s->d_part_res;
  a.update = update;
  return a;
}

static ScNodeArgs sc_node_args(const ipm_sc* s, int init) {
  ScNodeArgs n;
  n.Q = s->Q;
  n.n_parts = s->grid_x;
  n.init = init;
  n.steady = !(s->prob.t_end > 0.0);
  n.h = s->h;
  n.cfl = s->prob.cfl;
  n.t_end = s->prob.t_end;
  n.tol = s->tol;
  n.part_smax = s->d_part_smax;
  n.part_res = s->d_part_res;
  n.fixed_smax = s->d_fixed;
  n.t = s->d_t;
  n.steps = s->d_steps;
  n.res = s->d_res;
  n.dt = s->d_dt;
  n.n_active = s->d_active;
  return n;
}

static cudaError_t sc_launch_step(const ipm_sc* s, int from, int update) {
  const ScStepArgs a = sc_step_args(s, from, update);
  const dim3 grid(s->grid_x, s->grid_y);
  if (s->phys == PHYS_BURGERS) k_sc_step<PHYS_BURGERS, 1><<<grid, SC_T, 0, s->stream>>>(a);
  else if (s->phys == PHYS_EULER1D) k_sc_step<PHYS_EULER1D, 3><<<grid, SC_T, 0, s->stream>>>(a);
  else k_sc_step<PHYS_EULER2D, 4><<<grid, SC_T, 0, s->stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !update) return e;
  k_sc_nodes<<<1, 256, 0, s->stream>>>(sc_node_args(s, 0));
  return cudaGetLastError();
}

static void sc_free(ipm_sc* s) {
  if (!s) return;
  for (auto& g : s->exec)
    if (g) cudaGraphExecDestroy(g);
  for (auto& e : s->ev)
    if (e) cudaEventDestroy(e);
  void* ptrs[] = {s->d_u[0], s->d_u[1], s->d_PhiT, s->d_w, s->d_nodes, s->d_area, s->d_xf, s->d_yf,
                  s->d_part_smax, s->d_part_res, s->d_fixed, s->d_t, s->d_res, s->d_dt, s->d_steps, s->d_active,
                  s->d_ghosts};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (s->h_active) cudaFreeHost(s->h_active);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

static ipm_status sc_stats(ipm_sc* s, ipm_sc_stats* out, float elapsed_ms) {
  if (!out) return IPM_OK;
  std::vector<double> t(s->Q), r(s->Q);
  std::vector<long long> n(s->Q);
  SC_CK(s, cudaMemcpyAsync(t.data(), s->d_t, s->Q * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  SC_CK(s, cudaMemcpyAsync(r.data(), s->d_res, s->Q * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  SC_CK(s, cudaMemcpyAsync(n.data(), s->d_steps, s->Q * sizeof(long long), cudaMemcpyDeviceToHost, s->stream));
  SC_CK(s, cudaStreamSynchronize(s->stream));
  std::memset(out, 0, sizeof(*out));
  out->steps = s->steps;
  out->active_nodes = s->active;
  out->t_min = *std::min_element(t.begin(), t.end());
  out->t_max = *std::max_element(t.begin(), t.end());
  out->max_node_steps = *std::max_element(n.begin(), n.end());
  double rm = 0.0;
  for (double v : r) rm = std::isfinite(v) ? std::max(rm, v) : rm;
  out->residual_max = rm;
  out->elapsed_ms = elapsed_ms;
  return IPM_OK;
}

extern "C" {

ipm_status ipm_sc_init(const ipm_problem* problem, const ipm_basis* basis, const ipm_quadrature* quad,
                       double steady_tol, ipm_sc** out) {
  if (!problem || !basis || !quad || !out) return sc_fail(nullptr, IPM_EINVAL, "ipm_sc_init: null argument");
  *out = nullptr;
  if (const char* why = check_problem(problem, basis, quad))
    return sc_fail(nullptr, IPM_EINVAL, std::string("ipm_sc_init: ") + why);
  if (!(problem->t_end > 0.0) && !(steady_tol > 0.0))
    return sc_fail(nullptr, IPM_EINVAL, "ipm_sc_init: a steady run (t_end = 0) needs steady_tol > 0");
  ipm_sc* s = new ipm_sc();
  s->prob = *problem;
  s->tol = steady_tol;
  s->is2d = problem->kind == IPM_EULER_2D;
  s->m = problem->kind == IPM_BURGERS_1D ? 1 : (s->is2d ? 4 : 3);
  s->phys = problem->kind == IPM_BURGERS_1D ? PHYS_BURGERS : (s->is2d ? PHYS_EULER2D : PHYS_EULER1D);
  if (quad->kind == IPM_QUAD_CC_NESTED) {
    // the Clenshaw-Curtis rule of cc_level[0] (or the default level for the basis degree), as the
    // paper's collocation runs use
    int k = 0;
    if (const char* why = cc_levels(quad, basis->total_degree, 1, &k)) {
      delete s;
      return sc_fail(nullptr, IPM_EINVAL, std::string("ipm_sc_init: ") + why);
    }
    std::vector<std::vector<double>> lw;
    build_tables_cc(basis->p, basis->total_degree, k, s->tab, lw);
  } else {
    build_tables(basis->p, basis->total_degree, quad->n_per_dim, s->tab);
  }
  s->Q = s->tab.Q;
  s->N = s->tab.N;
  s->n_interior = s->is2d ? problem->nx * problem->ny : problem->nx;
  s->n_cells = s->is2d ? (problem->nx + 2) * (problem->ny + 2) : problem->nx + 2;
  if (s->is2d) {
    build_mesh2d(*problem, s->mesh);
    s->h = s->mesh.h_min;
  } else {
    s->h = (problem->x_hi - problem->x_lo) / problem->nx;
  }
  s->grid_y = (s->Q + 31) / 32;
  {
    int dev = 0, n_sm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    s->ch = 8;
    while (s->ch > 1 && (long long)((s->n_interior + s->ch - 1) / s->ch) * s->grid_y < 8LL * n_sm) s->ch /= 2;
  }
  s->grid_x = (s->n_interior + SC_W * s->ch - 1) / (SC_W * s->ch);
  // Dirichlet ghost cells (the ghost layer of every Dirichlet side, corners excluded)
  std::vector<int> ghosts;
  const int nx = problem->nx, ny = problem->ny;
  if (s->is2d) {
    for (int j = 0; j < ny; ++j) {
      if (problem->bc_left == IPM_BC_DIRICHLET) ghosts.push_back((j + 1) * (nx + 2));
      if (problem->bc_right == IPM_BC_DIRICHLET) ghosts.push_back((j + 1) * (nx + 2) + nx + 1);
    }
    for (int i = 0; i < nx; ++i) {
      if (problem->bc_bottom == IPM_BC_DIRICHLET) ghosts.push_back(i + 1);
      if (problem->bc_top == IPM_BC_DIRICHLET) ghosts.push_back((ny + 1) * (nx + 2) + i + 1);
    }
  } else {
    if (problem->bc_left == IPM_BC_DIRICHLET) ghosts.push_back(0);
    if (problem->bc_right == IPM_BC_DIRICHLET) ghosts.push_back(nx + 1);
  }
  const size_t nstate = (size_t)s->n_cells * s->m * s->Q;
  auto fail_free = [&](ipm_status st) {
    set_global_error(s->err);
    sc_free(s);
    return st;
  };
#define SC_INIT_CK(call)                                                                                \
  do {                                                                                                  \
    cudaError_t e_ = (call);                                                                            \
    if (e_ != cudaSuccess) {                                                                            \
      cudaGetLastError();                                                                               \
      s->err = std::string("ipm_sc_init: ") + #call + ": " + cudaGetErrorString(e_);                   \
      return fail_free(e_ == cudaErrorMemoryAllocation ? IPM_ENOMEM : IPM_ECUDA);                      \
    }                                                                                                   \
  } while (0)
  SC_INIT_CK(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
  SC_INIT_CK(cudaEventCreate(&s->ev[0]));
  SC_INIT_CK(cudaEventCreate(&s->ev[1]));
  SC_INIT_CK(cudaMalloc(&s->d_u[0], nstate * sizeof(double)));
  SC_INIT_CK(cudaMalloc(&s->d_u[1], nstate * sizeof(double)));
  SC_INIT_CK(sc_upload(&s->d_PhiT, s->tab.PhiT));
  SC_INIT_CK(sc_upload(&s->d_w, s->tab.w));
  SC_INIT_CK(sc_upload(&s->d_nodes, s->tab.nodes));
  if (s->is2d) {
    SC_INIT_CK(sc_upload(&s->d_area, s->mesh.area));
    SC_INIT_CK(sc_upload(&s->d_xf, s->mesh.xf));
    SC_INIT_CK(sc_upload(&s->d_yf, s->mesh.yf));
  }
  SC_INIT_CK(sc_upload(&s->d_ghosts, ghosts));
  const size_t parts = (size_t)s->grid_x * s->Q;
  SC_INIT_CK(cudaMalloc(&s->d_part_smax, parts * sizeof(double)));
  SC_INIT_CK(cudaMalloc(&s->d_part_res, parts * sizeof(double)));
  SC_INIT_CK(cudaMalloc(&s->d_fixed, s->Q * sizeof(double)));
  SC_INIT_CK(cudaMalloc(&s->d_t, s->Q * sizeof(double)));
  SC_INIT_CK(cudaMalloc(&s->d_res, s->Q * sizeof(double)));
  SC_INIT_CK(cudaMalloc(&s->d_dt, s->Q * sizeof(double)));
  SC_INIT_CK(cudaMalloc(&s->d_steps, s->Q * sizeof(long long)));
  SC_INIT_CK(cudaMalloc(&s->d_active, sizeof(int)));
  SC_INIT_CK(cudaMallocHost(&s->h_active, sizeof(int)));
  // initial states, Dirichlet ghost speeds, initial partials and the first time steps
  ScInitArgs ia;
  ia.ic1 = ic1d_params(*problem);
  ia.ic2 = s->is2d ? ic2d_params(*problem) : IC2D();
  ia.nodes = s->d_nodes;
  ia.p = basis->p;
  ia.Q = s->Q;
  ia.n_cells = s->n_cells;
  ia.nx = nx;
  ia.bc_left = problem->bc_left;
  ia.bc_right = problem->bc_right;
  ia.u0 = s->d_u[0];
  ia.u1 = s->d_u[1];
  const int ig = (int)std::min<size_t>(((size_t)s->n_cells * s->Q + 255) / 256, 8192);
  if (s->phys == PHYS_BURGERS) {
    k_sc_init<PHYS_BURGERS, 1><<<ig, 256, 0, s->stream>>>(ia);
    k_sc_fixed<PHYS_BURGERS, 1><<<(s->Q + 127) / 128, 128, 0, s->stream>>>(s->d_u[0], s->d_ghosts, (int)ghosts.size(),
                                                                             s->Q, problem->gamma, s->d_fixed);
  } else if (s->phys == PHYS_EULER1D) {
    k_sc_init<PHYS_EULER1D, 3><<<ig, 256, 0, s->stream>>>(ia);
    k_sc_fixed<PHYS_EULER1D, 3><<<(s->Q + 127) / 128, 128, 0, s->stream>>>(s->d_u[0], s->d_ghosts, (int)ghosts.size(),
                                                                              s->Q, problem->gamma, s->d_fixed);
  } else {
    k_sc_init<PHYS_EULER2D, 4><<<ig, 256, 0, s->stream>>>(ia);
    k_sc_fixed<PHYS_EULER2D, 4><<<(s->Q + 127) / 128, 128, 0, s->stream>>>(s->d_u[0], s->d_ghosts, (int)ghosts.size(),
                                                                              s->Q, problem->gamma, s->d_fixed);
  }
  SC_INIT_CK(cudaGetLastError());
  SC_INIT_CK(sc_launch_step(s, 0, 0));
  k_sc_nodes<<<1, 256, 0, s->stream>>>(sc_node_args(s, 1));
  SC_INIT_CK(cudaGetLastError());
  SC_INIT_CK(cudaMemcpyAsync(s->h_active, s->d_active, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  SC_INIT_CK(cudaStreamSynchronize(s->stream));
  s->active = *s->h_active;
#undef SC_INIT_CK
  *out = s;
  return IPM_OK;
}

ipm_status ipm_sc_step(ipm_sc* s, ipm_sc_stats* stats) {
  NvtxRange nvtx_("ipm_sc_step");
  if (!s) return sc_fail(nullptr, IPM_EINVAL, "ipm_sc_step: null handle");
  SC_CK(s, cudaEventRecord(s->ev[0], s->stream));
  SC_CK(s, sc_launch_step(s, s->cur, 1));
  SC_CK(s, cudaEventRecord(s->ev[1], s->stream));
  s->cur ^= 1;
  ++s->steps;
  SC_CK(s, cudaMemcpyAsync(s->h_active, s->d_active, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  SC_CK(s, cudaStreamSynchronize(s->stream));
  s->active = *s->h_active;
  float ms = 0.f;
  SC_CK(s, cudaEventElapsedTime(&ms, s->ev[0], s->ev[1]));
  return sc_stats(s, stats, ms);
}

ipm_status ipm_sc_run(ipm_sc* s, int64_t max_steps, ipm_sc_stats* stats) {
  NvtxRange nvtx_("ipm_sc_run");
  if (!s) return sc_fail(nullptr, IPM_EINVAL, "ipm_sc_run: null handle");
  SC_CK(s, cudaEventRecord(s->ev[0], s->stream));
  while (s->active > 0 && s->steps < max_steps) {
    if (max_steps - s->steps >= SC_GRAPH_STEPS) {
      if (!s->exec[s->cur]) {
        cudaGraph_t g = nullptr;
        SC_CK(s, cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < SC_GRAPH_STEPS && e == cudaSuccess; ++k) e = sc_launch_step(s, s->cur ^ (k & 1), 1);
        cudaError_t e2 = cudaStreamEndCapture(s->stream, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&s->exec[s->cur], g, 0);
        if (g) cudaGraphDestroy(g);
        SC_CK(s, e);
      }
      SC_CK(s, cudaGraphLaunch(s->exec[s->cur], s->stream));
      s->steps += SC_GRAPH_STEPS;
    } else {
      SC_CK(s, sc_launch_step(s, s->cur, 1));
      s->cur ^= 1;
      ++s->steps;
    }
    SC_CK(s, cudaMemcpyAsync(s->h_active, s->d_active, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    SC_CK(s, cudaStreamSynchronize(s->stream));
    s->active = *s->h_active;
  }
  SC_CK(s, cudaEventRecord(s->ev[1], s->stream));
  SC_CK(s, cudaEventSynchronize(s->ev[1]));
  float ms = 0.f;
  SC_CK(s, cudaEventElapsedTime(&ms, s->ev[0], s->ev[1]));
  return sc_stats(s, stats, ms);
}

ipm_status ipm_sc_get_nodal(ipm_sc* s, double* host, size_t count) {
  if (!s || !host) return sc_fail(s, IPM_EINVAL, "ipm_sc_get_nodal: null argument");
  const size_t n = (size_t)s->n_cells * s->Q * s->m;
  if (count != n) return sc_fail(s, IPM_EINVAL, "ipm_sc_get_nodal: count must be cells * nodes * variables");
  std::vector<double> tmp(n);
  SC_CK(s, cudaMemcpyAsync(tmp.data(), s->d_u[s->cur], n * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  SC_CK(s, cudaStreamSynchronize(s->stream));
  // [cell][variable][node] -> [cell][node][variable]
  for (int c = 0; c < s->n_cells; ++c)
    for (int k = 0; k < s->m; ++k)
      for (int q = 0; q < s->Q; ++q)
        host[((size_t)c * s->Q + q) * s->m + k] = tmp[((size_t)c * s->m + k) * s->Q + q];
  return IPM_OK;
}

ipm_status ipm_sc_get_moments(ipm_sc* s, double* host, size_t count) {
  if (!s || !host) return sc_fail(s, IPM_EINVAL, "ipm_sc_get_moments: null argument");
  const size_t n = (size_t)s->n_cells * s->N * s->m;
  if (count != n) return sc_fail(s, IPM_EINVAL, "ipm_sc_get_moments: count must be cells * moments * variables");
  double* d = nullptr;
  SC_CK(s, cudaMallocAsync(&d, n * sizeof(double), s->stream));
  const int grid = std::min(s->n_cells, 8192);
  const double* u = s->d_u[s->cur];
  if (s->m == 1) k_sc_moments<1><<<grid, 256, 0, s->stream>>>(u, s->d_PhiT, s->d_w, s->N, s->Q, s->n_cells, d);
  else if (s->m == 3) k_sc_moments<3><<<grid, 256, 0, s->stream>>>(u, s->d_PhiT, s->d_w, s->N, s->Q, s->n_cells, d);
  else k_sc_moments<4><<<grid, 256, 0, s->stream>>>(u, s->d_PhiT, s->d_w, s->N, s->Q, s->n_cells, d);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, d, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  cudaFreeAsync(d, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  SC_CK(s, e);
  return IPM_OK;
}

ipm_status ipm_sc_get_node_info(ipm_sc* s, int64_t* steps, double* t, double* residual, size_t count) {
  if (!s) return sc_fail(nullptr, IPM_EINVAL, "ipm_sc_get_node_info: null handle");
  if (count != (size_t)s->Q) return sc_fail(s, IPM_EINVAL, "ipm_sc_get_node_info: count must be the node count");
  static_assert(sizeof(long long) == sizeof(int64_t), "64-bit counters");
  if (steps) SC_CK(s, cudaMemcpyAsync(steps, s->d_steps, count * sizeof(int64_t), cudaMemcpyDeviceToHost, s->stream));
  if (t) SC_CK(s, cudaMemcpyAsync(t, s->d_t, count * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  if (residual) SC_CK(s, cudaMemcpyAsync(residual, s->d_res, count * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  SC_CK(s, cudaStreamSynchronize(s->stream));
  return IPM_OK;
}

ipm_status ipm_sc_get_dims(const ipm_sc* s, int* n_cells, int* n_nodes, int* n_moments, int* n_vars) {
  if (!s) return IPM_EINVAL;
  if (n_cells) *n_cells = s->n_cells;
  if (n_nodes) *n_nodes = s->Q;
  if (n_moments) *n_moments = s->N;
  if (n_vars) *n_vars = s->m;
  return IPM_OK;
}

const char* ipm_sc_last_error(const ipm_sc* s) { return s ? s->err.c_str() : ipm_last_error(nullptr); }

void ipm_sc_destroy(ipm_sc* s) {
  if (s && s->stream) cudaStreamSynchronize(s->stream);
  sc_free(s);
}

}  // extern "C"
