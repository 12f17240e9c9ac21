// update2d.cu -- 2-D Euler (Sec. 7): mesh geometry, initial data and the kinetic-flux moment update
// on structured quadrilateral meshes.
//
// Moment update of an interior cell c (Eq. momentIterationFunction in quadrature form, Eq.
// momentUpQuadrature, with the divergence theorem over the cell's four faces):
//   u_c^{n+1} = sum_k w_k [u_k^(c) - dt/A_c (L_r g_r - L_l g_l + L_t g_t - L_b g_b)] phi(xi_k),
// g the local Lax-Friedrichs (Rusanov) flux across a face, node by node:
//   g(u_a, u_b; n) = (F(u_a).n + F(u_b).n)/2 - a/2 (u_b - u_a),  a = max(|v_a.n| + c_a, |v_b.n| + c_b),
// with u_a behind and u_b ahead of the face normal (normals point to increasing i or j).
// Sides: periodic wraps; outflow uses the cell's own nodal state; Dirichlet ghosts keep the nodal
// states of their duals converged at init; a slip wall reflects the momentum about the face normal.
// dt = CFL h / s_max (h = min area / longest face, s_max from the Newton kernel's atomic maximum),
// clipped to t_end on Algorithm-1 steps.
#include <cmath>

#include "ic.cuh"
#include "ipm_host.h"

namespace ipm {

constexpr int T2 = 256;
constexpr int W2 = T2 / 32;

__global__ void __launch_bounds__(T2) k_update2d(Update2DArgs a) {
  extern __shared__ __align__(16) double s_v[];     // [4][Q] w * integrand, then [W2][N 4] partial sums
  constexpr int M = 4;
  const int N = a.tab.N, Q = a.tab.Q, NM = N * M;
  const int nx = a.mesh.nx, ny = a.mesh.ny;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double dt = a.dt_override;
  if (!(dt > 0.0)) {
    const double smax = __longlong_as_double((long long)a.sc->smax_bits);
    dt = a.cfl * a.mesh.h_min / smax;
    if (a.clip && a.t_end > 0.0 && a.sc->t + dt > a.t_end) dt = a.t_end - a.sc->t;
  }
  if (blockIdx.x == 0 && tid == 0) a.sc->dt = dt > 0.0 ? dt : 0.0;
  if (!(dt > 0.0)) return;
  const double* __restrict__ w = a.tab.w;
  const double* __restrict__ Phi = a.tab.Phi;
  const int MQ = M * Q;
  const double g = a.gamma;
  double* s_part = s_v + MQ;

  for (int cidx = blockIdx.x; cidx < nx * ny; cidx += gridDim.x) {
    const int i = cidx % nx, j = cidx / nx;
    const int c = cell2d(i, j, nx);
    // adaptive meshes: the new level (k_next_levels) sets the moments kept and, with a rule per level,
    // the nodes and weights of the update's quadrature (Eq. adaptiveFVUpdate)
    int lev_new = 0, n_new = N, Qn = Q;
    const double* wn = w;
    if (a.level) {
      lev_new = a.level_next[c];
      n_new = a.lev_n[lev_new];
      if (a.lev_w) {
        Qn = a.lev_q[lev_new];
        wn = a.lev_w + (size_t)lev_new * Q;
      }
    }
    const double area = a.mesh.area[(size_t)j * nx + i];
    const double* xl = a.mesh.xf + ((size_t)j * (nx + 1) + i) * 3;
    const double* xr = xl + 3;
    const double* yb = a.mesh.yf + ((size_t)j * nx + i) * 3;
    const double* yt = a.mesh.yf + ((size_t)(j + 1) * nx + i) * 3;
    const int nl = i > 0 ? cell2d(i - 1, j, nx) : outside(a.bc[0], cell2d(nx - 1, j, nx), cell2d(-1, j, nx));
    const int nr = i < nx - 1 ? cell2d(i + 1, j, nx) : outside(a.bc[1], cell2d(0, j, nx), cell2d(nx, j, nx));
    const int nb = j > 0 ? cell2d(i, j - 1, nx) : outside(a.bc[2], cell2d(i, ny - 1, nx), cell2d(i, -1, nx));
    const int nt = j < ny - 1 ? cell2d(i, j + 1, nx) : outside(a.bc[3], cell2d(i, 0, nx), cell2d(i, ny, nx));
    const double r = dt / area;
    for (int q = tid; q < Qn; q += T2) {
      double uc[M], un[M], f[M], acc[M];
      const double* ucg = a.unode + (size_t)c * MQ;
#pragma unroll
      for (int k = 0; k < M; ++k) {
        uc[k] = ucg[k * Q + q];
        acc[k] = 0.0;
      }
      // faces: (neighbour, normal, sign): flux behind->ahead; left/bottom: neighbour behind
      const int nbr[4] = {nl, nr, nb, nt};
      const double* fg[4] = {xl, xr, yb, yt};
#pragma unroll
      for (int fa = 0; fa < 4; ++fa) {
        const double nxn = fg[fa][0], nyn = fg[fa][1], L = fg[fa][2];
        const int o = nbr[fa];
        if (o >= 0) {
          const double* ug = a.unode + (size_t)o * MQ;
#pragma unroll
          for (int k = 0; k < M; ++k) un[k] = ug[k * Q + q];
        } else if (o == -1) {
#pragma unroll
          for (int k = 0; k < M; ++k) un[k] = uc[k];
        } else {
          reflect(uc, nxn, nyn, un);
        }
        const bool ahead = (fa & 1) != 0;            // right and top faces: the neighbour is ahead
        if (ahead) rusanov2d(uc, un, nxn, nyn, g, f);
        else rusanov2d(un, uc, nxn, nyn, g, f);
        const double sL = ahead ? L : -L;
#pragma unroll
        for (int k = 0; k < M; ++k) acc[k] = fma(sL, f[k], acc[k]);
      }
      const double wq = wn[q];
#pragma unroll
      for (int k = 0; k < M; ++k) s_v[k * Q + q] = wq * fma(-r, acc[k], uc[k]);
    }
    __syncthreads();
    double* out = a.uhat + (size_t)c * NM;
    const double old00 = out[0];
    // projection onto the new level: warp k sums the nodes [k qw, (k+1) qw) for every entry (lanes over
    // entries), then the warps' partial sums are added in warp order
    const int NMn = n_new * M;
    const int qw = (Qn + W2 - 1) / W2;
    const int q_lo = min(Qn, warp * qw), q_hi = min(Qn, q_lo + qw);
    for (int rr = lane; rr < NMn; rr += 32) {
      const int ii = rr / M, k = rr - ii * M;
      double acc = 0.0;
      for (int q = q_lo; q < q_hi; ++q) acc = fma(Phi[(size_t)q * N + ii], s_v[k * Q + q], acc);
      s_part[warp * NM + rr] = acc;
    }
    __syncthreads();
    for (int rr = tid; rr < NM; rr += T2) {
      if (rr >= NMn) {                                     // beyond the new level: moments and duals are zero
        out[rr] = 0.0;
        a.lam[(size_t)c * NM + rr] = 0.0;
        continue;
      }
      double v = 0.0;
#pragma unroll
      for (int k = 0; k < W2; ++k) v += s_part[k * NM + rr];
      out[rr] = v;
    }
    __syncthreads();
    if (tid == 0 && a.cell_resid) a.cell_resid[c] = area * fabs(out[0] - old00);
    if (tid == 0 && a.level) a.level[c] = lev_new;
    __syncthreads();
  }
}

// New refinement levels (Algorithm 3, DetermineRefinementLevel) from the smoothness indicator of the
// density moments u_hat^n at each interior cell's level (Eq. errorIndicator): keep inside
// [delta_lo, delta_hi], one level down below, one level up above, clamped to 0 .. min(levels - 1, cap).
// One warp per interior cell.
__global__ void k_next_levels(Update2DArgs a) {
  constexpr int M = 4;
  const int NM = a.tab.N * M, nx = a.mesh.nx, ny = a.mesh.ny;
  const int lane = threadIdx.x & 31;
  const int wk = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (wk >= nx * ny) return;
  const int c = cell2d(wk % nx, wk / nx, nx);
  const double* u = a.uhat + (size_t)c * NM;
  const int lev = a.level[c];
  const int n_lev = a.lev_n[lev], n_prv = a.lev_prev[lev];
  double top = 0.0, tot = 0.0;
  for (int ii = lane; ii < n_lev; ii += 32) {
    const double v = u[ii * M];
    tot = fma(v, v, tot);
    if (ii >= n_prv) top = fma(v, v, top);
  }
  top = warp_sum(top);
  tot = warp_sum(tot);
  const double S = top / tot;
  int lev_new = S < a.delta_lo ? lev - 1 : (S > a.delta_hi ? lev + 1 : lev);
  lev_new = min(max(lev_new, 0), min(a.n_levels - 1, a.sc->level_cap));
  if (lane == 0) a.level_next[c] = lev_new;
}

// Per-level rules: the nodes each interior cell's nodal states must cover, the largest rule among the new
// levels of the cell and of the cells its faces read (the paper's coarser neighbour evaluated at the
// finer nodes). Dirichlet ghosts keep all nodes. One thread per interior cell.
__global__ void k_eval_q(Update2DArgs a) {
  const int nx = a.mesh.nx, ny = a.mesh.ny;
  const int wk = blockIdx.x * blockDim.x + threadIdx.x;
  if (wk >= nx * ny) return;
  const int i = wk % nx, j = wk / nx;
  const int c = cell2d(i, j, nx);
  const int nb[4] = {i > 0 ? cell2d(i - 1, j, nx) : outside(a.bc[0], cell2d(nx - 1, j, nx), cell2d(-1, j, nx)),
                     i < nx - 1 ? cell2d(i + 1, j, nx) : outside(a.bc[1], cell2d(0, j, nx), cell2d(nx, j, nx)),
                     j > 0 ? cell2d(i, j - 1, nx) : outside(a.bc[2], cell2d(i, ny - 1, nx), cell2d(i, -1, nx)),
                     j < ny - 1 ? cell2d(i, j + 1, nx) : outside(a.bc[3], cell2d(i, 0, nx), cell2d(i, ny, nx))};
  int e = a.lev_q[a.level_next[c]];
  for (int f = 0; f < 4; ++f)
    if (nb[f] >= 0) e = max(e, a.lev_q[a.level_next[nb[f]]]);
  a.q_eval[c] = e;
}

cudaError_t launch_next_levels(const Update2DArgs& a, cudaStream_t s) {
  const int n = a.mesh.nx * a.mesh.ny;
  k_next_levels<<<(n + 7) / 8, 256, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && a.q_eval) {
    k_eval_q<<<(n + 255) / 256, 256, 0, s>>>(a);
    e = cudaGetLastError();
  }
  return e;
}

// Initial refinement levels (adaptive meshes): from the finest projection, lower the level of every
// cell one step at a time while its indicator is below delta_lo, then zero the moments and duals
// beyond the level. One warp per cell.
__global__ void k_init_levels(Update2DArgs a, int n_cells) {
  constexpr int M = 4;
  const int N = a.tab.N, NM = N * M;
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (c >= n_cells) return;
  const double* u = a.uhat + (size_t)c * NM;
  int lev = a.n_levels - 1;
  for (int k = 0; k < a.n_levels; ++k) {
    const int nl = a.lev_n[lev], np = a.lev_prev[lev];
    double top = 0.0, tot = 0.0;
    for (int ii = lane; ii < nl; ii += 32) {
      const double v = u[ii * M];
      tot = fma(v, v, tot);
      if (ii >= np) top = fma(v, v, top);
    }
    top = warp_sum(top);
    tot = warp_sum(tot);
    if (lev > 0 && top / tot < a.delta_lo) --lev;
  }
  const int n = a.lev_n[lev];
  for (int r = n * M + lane; r < NM; r += 32) {
    a.uhat[(size_t)c * NM + r] = 0.0;
    a.lam[(size_t)c * NM + r] = 0.0;
  }
  if (lane == 0) a.level[c] = lev;
}

// Lower every interior level above cap to cap and zero the moments and duals beyond it (Algorithm 4:
// the maximal level of a retardation stage). One warp per interior cell.
__global__ void k_cap_levels(Update2DArgs a, int cap) {
  constexpr int M = 4;
  const int N = a.tab.N, NM = N * M, nx = a.mesh.nx, ny = a.mesh.ny;
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (w >= nx * ny) return;
  const int c = cell2d(w % nx, w / nx, nx);
  const int lev = a.level[c];
  if (lev <= cap) return;
  const int n = a.lev_n[cap];
  for (int r = n * M + lane; r < NM; r += 32) {
    a.uhat[(size_t)c * NM + r] = 0.0;
    a.lam[(size_t)c * NM + r] = 0.0;
  }
  if (lane == 0) a.level[c] = cap;
}

cudaError_t launch_cap_levels(const Update2DArgs& a, int cap, cudaStream_t s) {
  const int n = a.mesh.nx * a.mesh.ny;
  k_cap_levels<<<(n + 7) / 8, 256, 0, s>>>(a, cap);
  return cudaGetLastError();
}

cudaError_t launch_init_levels(const Update2DArgs& a, int n_cells, cudaStream_t s) {
  k_init_levels<<<(n_cells + 7) / 8, 256, 0, s>>>(a, n_cells);
  return cudaGetLastError();
}

// The same update with one warp per cell (8 cells per CTA) for small node counts: lanes over nodes
// for the fluxes, lanes over moments for the projection, no block barriers.
constexpr int UPD_WARPS = 8;

__global__ void __launch_bounds__(256) k_update2d_warp(Update2DArgs a) {
  extern __shared__ __align__(16) double s_all[];
  constexpr int M = 4;
  const int N = a.tab.N, Q = a.tab.Q, NM = N * M;
  const int nx = a.mesh.nx, ny = a.mesh.ny;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* s_v = s_all + (size_t)warp * M * Q;
  double dt = a.dt_override;
  if (!(dt > 0.0)) {
    const double smax = __longlong_as_double((long long)a.sc->smax_bits);
    dt = a.cfl * a.mesh.h_min / smax;
    if (a.clip && a.t_end > 0.0 && a.sc->t + dt > a.t_end) dt = a.t_end - a.sc->t;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) a.sc->dt = dt > 0.0 ? dt : 0.0;
  if (!(dt > 0.0)) return;
  const double* __restrict__ w = a.tab.w;
  const double* __restrict__ PhiT = a.tab.PhiT;
  const int MQ = M * Q;
  const double g = a.gamma;
  for (int cidx = blockIdx.x * UPD_WARPS + warp; cidx < nx * ny; cidx += gridDim.x * UPD_WARPS) {
    const int i = cidx % nx, j = cidx / nx;
    const int c = cell2d(i, j, nx);
    int lev_new = 0, n_new = N, Qn = Q;
    const double* wn = w;
    if (a.level) {
      lev_new = a.level_next[c];
      n_new = a.lev_n[lev_new];
      if (a.lev_w) {
        Qn = a.lev_q[lev_new];
        wn = a.lev_w + (size_t)lev_new * Q;
      }
    }
    const double area = a.mesh.area[(size_t)j * nx + i];
    const double* xl = a.mesh.xf + ((size_t)j * (nx + 1) + i) * 3;
    const double* xr = xl + 3;
    const double* yb = a.mesh.yf + ((size_t)j * nx + i) * 3;
    const double* yt = a.mesh.yf + ((size_t)(j + 1) * nx + i) * 3;
    const int nl = i > 0 ? cell2d(i - 1, j, nx) : outside(a.bc[0], cell2d(nx - 1, j, nx), cell2d(-1, j, nx));
    const int nr = i < nx - 1 ? cell2d(i + 1, j, nx) : outside(a.bc[1], cell2d(0, j, nx), cell2d(nx, j, nx));
    const int nb = j > 0 ? cell2d(i, j - 1, nx) : outside(a.bc[2], cell2d(i, ny - 1, nx), cell2d(i, -1, nx));
    const int nt = j < ny - 1 ? cell2d(i, j + 1, nx) : outside(a.bc[3], cell2d(i, 0, nx), cell2d(i, ny, nx));
    const double r = dt / area;
    for (int q = lane; q < Qn; q += 32) {
      double uc[M], un[M], f[M], acc[M];
      const double* ucg = a.unode + (size_t)c * MQ;
#pragma unroll
      for (int k = 0; k < M; ++k) {
        uc[k] = ucg[k * Q + q];
        acc[k] = 0.0;
      }
      const int nbr[4] = {nl, nr, nb, nt};
      const double* fg[4] = {xl, xr, yb, yt};
#pragma unroll
      for (int fa = 0; fa < 4; ++fa) {
        const double nxn = fg[fa][0], nyn = fg[fa][1], L = fg[fa][2];
        const int o = nbr[fa];
        if (o >= 0) {
          const double* ug = a.unode + (size_t)o * MQ;
#pragma unroll
          for (int k = 0; k < M; ++k) un[k] = ug[k * Q + q];
        } else if (o == -1) {
#pragma unroll
          for (int k = 0; k < M; ++k) un[k] = uc[k];
        } else {
          reflect(uc, nxn, nyn, un);
        }
        const bool ahead = (fa & 1) != 0;
        if (ahead) rusanov2d(uc, un, nxn, nyn, g, f);
        else rusanov2d(un, uc, nxn, nyn, g, f);
        const double sL = ahead ? L : -L;
#pragma unroll
        for (int k = 0; k < M; ++k) acc[k] = fma(sL, f[k], acc[k]);
      }
      const double wq = wn[q];
#pragma unroll
      for (int k = 0; k < M; ++k) s_v[k * Q + q] = wq * fma(-r, acc[k], uc[k]);
    }
    __syncwarp();
    double* out = a.uhat + (size_t)c * NM;
    const double old00 = out[0];
    for (int rr = lane; rr < NM; rr += 32) {
      const int ii = rr / M, k = rr - ii * M;
      double v = 0.0;
      if (ii < n_new) {
        for (int q = 0; q < Qn; ++q) v = fma(PhiT[(size_t)ii * Q + q], s_v[k * Q + q], v);
      } else {
        a.lam[(size_t)c * NM + rr] = 0.0;
      }
      out[rr] = v;
    }
    __syncwarp();
    if (lane == 0 && a.cell_resid) a.cell_resid[c] = area * fabs(out[0] - old00);
    if (lane == 0 && a.level) a.level[c] = lev_new;
    __syncwarp();
  }
}

// the warp variant when a warp's slice of node values is small; else one CTA per cell
static bool update2d_use_warp(int Q) { return Q <= 64; }

static size_t update2d_smem(int N, int Q) { return ((size_t)4 * Q + (size_t)W2 * N * 4) * sizeof(double); }

cudaError_t prepare_update2d(int N, int Q) {
  if (update2d_use_warp(Q)) return raise_smem_limit(k_update2d_warp, (size_t)UPD_WARPS * 4 * Q * sizeof(double));
  return raise_smem_limit(k_update2d, update2d_smem(N, Q));
}

cudaError_t launch_update2d(const Update2DArgs& a, int grid, cudaStream_t s) {
  if (update2d_use_warp(a.tab.Q)) {
    const int cells = a.mesh.nx * a.mesh.ny;
    const int g = std::max(1, std::min((cells + UPD_WARPS - 1) / UPD_WARPS, 65535));
    k_update2d_warp<<<g, 32 * UPD_WARPS, (size_t)UPD_WARPS * 4 * a.tab.Q * sizeof(double), s>>>(a);
  } else {
    k_update2d<<<grid, T2, update2d_smem(a.tab.N, a.tab.Q), s>>>(a);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Initial data on every cell (ghosts included): nodal cell averages of the 2-D initial data,
// projected; initial duals = projection of grad s of the nodal averages.
// ------------------------------------------------------------------------------------------------
struct Init2DArgs {
  Tables tab;
  EntParams ent;
  IC2D ic;
  double* uhat;
  double* lam;
  const int* level;      // per-level projection (rule per level), or nullptr
  int lev_n[8], lev_q[8];
  const double* lev_w;
};

template <int ENT>
__global__ void __launch_bounds__(T2) k_init2d(Init2DArgs a) {
  extern __shared__ __align__(16) double sm[];
  constexpr int M = 4;
  const int N = a.tab.N, Q = a.tab.Q, P = a.tab.p, NM = N * M;
  double* s_u = sm;            // [M][Q] w * ubar
  double* s_e = sm + M * Q;    // [M][Q] w * grad s(ubar)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nx = a.ic.nx, ny = a.ic.ny, n_cells = (nx + 2) * (ny + 2);
  for (int c = blockIdx.x; c < n_cells; c += gridDim.x) {
    const int ii = c % (nx + 2), jj = c / (nx + 2);              // ghost-inclusive column and row
    int Nc = N, Qc = Q;
    const double* wc = a.tab.w;
    if (a.level) {
      const int l = a.level[c];
      Nc = a.lev_n[l];
      Qc = a.lev_q[l];
      wc = a.lev_w + (size_t)l * Q;
    }
    for (int q = tid; q < Qc; q += T2) {
      double xi[3] = {0.0, 0.0, 0.0};
      for (int d = 0; d < P; ++d) xi[d] = a.tab.nodes[(size_t)q * P + d];
      double ub[M], ge[M];
      ic2d_average(a.ic, ii, jj, xi, P, ub);
      entropy_gradient<ENT, M>(ub, a.ent, ge);
      const double wq = wc[q];
#pragma unroll
      for (int k = 0; k < M; ++k) {
        s_u[k * Q + q] = wq * ub[k];
        s_e[k * Q + q] = wq * ge[k];
      }
    }
    __syncthreads();
    for (int i = warp; i < N; i += W2) {
      double au[M], ae[M];
#pragma unroll
      for (int k = 0; k < M; ++k) au[k] = ae[k] = 0.0;
      for (int q = lane; q < (i < Nc ? Qc : 0); q += 32) {      // moments beyond the level stay zero
        const double ph = a.tab.PhiT[(size_t)i * Q + q];
#pragma unroll
        for (int k = 0; k < M; ++k) {
          au[k] = fma(ph, s_u[k * Q + q], au[k]);
          ae[k] = fma(ph, s_e[k * Q + q], ae[k]);
        }
      }
#pragma unroll
      for (int k = 0; k < M; ++k) {
        const double vu = warp_sum(au[k]), ve = warp_sum(ae[k]);
        if (lane == 0) {
          a.uhat[(size_t)c * NM + i * M + k] = vu;
          a.lam[(size_t)c * NM + i * M + k] = ve;
        }
      }
    }
    __syncthreads();
  }
}

cudaError_t launch_init2d(int ent, const Tables& tab, const EntParams& ent_p, const ipm_problem& prob, double* uhat,
                          double* lam, cudaStream_t s, const int* level, const int* lev_n, const int* lev_q,
                          const double* lev_w) {
  Init2DArgs a;
  a.tab = tab;
  a.ent = ent_p;
  a.ic = ic2d_params(prob);
  a.level = level;
  for (int l = 0; l < 8; ++l) {
    a.lev_n[l] = level ? lev_n[l] : 0;
    a.lev_q[l] = level ? lev_q[l] : 0;
  }
  a.lev_w = lev_w;
  a.uhat = uhat;
  a.lam = lam;
  const int n_cells = (prob.nx + 2) * (prob.ny + 2);
  const size_t smem = 2 * (size_t)4 * tab.Q * sizeof(double);
  const int grid = n_cells < 8192 ? n_cells : 8192;
  if (ent == ENT_EULER) {
    cudaError_t e = raise_smem_limit(k_init2d<ENT_EULER>, smem);
    if (e != cudaSuccess) return e;
    k_init2d<ENT_EULER><<<grid, T2, smem, s>>>(a);
  } else if (ent == ENT_QUADRATIC) {
    cudaError_t e = raise_smem_limit(k_init2d<ENT_QUADRATIC>, smem);
    if (e != cudaSuccess) return e;
    k_init2d<ENT_QUADRATIC><<<grid, T2, smem, s>>>(a);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Host: vertices of the mesh, cell areas (shoelace), face normals and lengths, h.
// ------------------------------------------------------------------------------------------------
void build_mesh2d(const ipm_problem& pr, Mesh2DHost& m) {
  const int nx = pr.nx, ny = pr.ny;
  std::vector<double> X((size_t)(nx + 1) * (ny + 1)), Y(X.size());
  auto V = [&](int i, int j) { return (size_t)i * (ny + 1) + j; };
  const double tr = std::tan(pr.ramp_deg * M_PI / 180.0);
  for (int i = 0; i <= nx; ++i) {
    const double x = pr.x_lo + (pr.x_hi - pr.x_lo) * i / nx;
    const double yb = pr.mesh_kind == IPM_MESH_RAMP && x > pr.ramp_x0 ? pr.y_lo + (x - pr.ramp_x0) * tr : pr.y_lo;
    for (int j = 0; j <= ny; ++j) {
      const double eta = (double)j / ny;
      X[V(i, j)] = x;
      Y[V(i, j)] = pr.mesh_kind == IPM_MESH_RAMP ? yb + (pr.y_hi - yb) * eta : pr.y_lo + (pr.y_hi - pr.y_lo) * eta;
    }
  }
  m.area.assign((size_t)nx * ny, 0.0);
  m.xf.assign((size_t)ny * (nx + 1) * 3, 0.0);
  m.yf.assign((size_t)(ny + 1) * nx * 3, 0.0);
  for (int j = 0; j < ny; ++j)
    for (int f = 0; f <= nx; ++f) {
      const double dx = X[V(f, j + 1)] - X[V(f, j)], dy = Y[V(f, j + 1)] - Y[V(f, j)];
      const double L = std::hypot(dx, dy);
      double* o = &m.xf[((size_t)j * (nx + 1) + f) * 3];
      o[0] = dy / L;
      o[1] = -dx / L;
      o[2] = L;
    }
  for (int g = 0; g <= ny; ++g)
    for (int i = 0; i < nx; ++i) {
      const double dx = X[V(i + 1, g)] - X[V(i, g)], dy = Y[V(i + 1, g)] - Y[V(i, g)];
      const double L = std::hypot(dx, dy);
      double* o = &m.yf[((size_t)g * nx + i) * 3];
      o[0] = -dy / L;
      o[1] = dx / L;
      o[2] = L;
    }
  m.h_min = 1e300;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const double x[4] = {X[V(i, j)], X[V(i + 1, j)], X[V(i + 1, j + 1)], X[V(i, j + 1)]};
      const double y[4] = {Y[V(i, j)], Y[V(i + 1, j)], Y[V(i + 1, j + 1)], Y[V(i, j + 1)]};
      double a = 0.0;
      for (int k = 0; k < 4; ++k) a += x[k] * y[(k + 1) % 4] - x[(k + 1) % 4] * y[k];
      a *= 0.5;
      m.area[(size_t)j * nx + i] = a;
      const double longest = std::max(std::max(m.xf[((size_t)j * (nx + 1) + i) * 3 + 2], m.xf[((size_t)j * (nx + 1) + i + 1) * 3 + 2]),
                                      std::max(m.yf[((size_t)j * nx + i) * 3 + 2], m.yf[((size_t)(j + 1) * nx + i) * 3 + 2]));
      m.h_min = std::min(m.h_min, a / longest);
    }
}

}  // namespace ipm
