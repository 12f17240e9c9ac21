// update.cu -- kinetic-flux moment update, initial data, boundary copies and per-step bookkeeping
// for 1-D meshes.
//
// Moment update c of an interior cell j (Eq. momentIterationFunction in the quadrature form of
// Eq. momentUpQuadrature):
//   u_j^{n+1} = sum_k w_k [u_k^(j) - dt/dx (g(u_k^(j), u_k^(j+1)) - g(u_k^(j-1), u_k^(j)))] phi(xi_k)
// with u_k^(j) the nodal states u_s(lambda_j^T phi(xi_k)) written by the Newton kernel and g the
// Lax-Friedrichs flux g(u_l, u_r) = (f(u_l) + f(u_r))/2 - dx/(2 dt) (u_r - u_l) (App. A).
// dt = CFL dx / max speed (the maximum the Newton kernel folded into StepScalars), clipped to t_end.
// Ghost neighbours are resolved through the boundary condition: outflow reads the cell itself,
// periodic the opposite end, Dirichlet the fixed ghost.
#include "ic.cuh"
#include "ipm_host.h"

namespace ipm {

constexpr int UT = 256;
constexpr int UWARPS = UT / 32;

__device__ __forceinline__ double step_dt(const Update1DArgs& a) {
  if (a.dt_override > 0.0) return a.dt_override;
  const double smax = __longlong_as_double((long long)a.sc->smax_bits);
  double dt = a.cfl * a.dx / smax;
  if (a.t_end > 0.0 && a.sc->t + dt > a.t_end) dt = a.t_end - a.sc->t;
  return dt;
}

template <int PHYS, int M>
__global__ void __launch_bounds__(UT) k_update1d(Update1DArgs a) {
  extern __shared__ __align__(16) double s_v[];     // [M][Q] integrand, then [UWARPS][N M] partial sums
  const int N = a.tab.N, Q = a.tab.Q, NM = N * M;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double dt = step_dt(a);
  if (blockIdx.x == 0 && tid == 0) a.sc->dt = dt > 0.0 ? dt : 0.0;
  if (!(dt > 0.0)) return;                                 // t reached t_end: nothing to do
  const double nu = a.dx / (2.0 * dt);
  const double r = dt / a.dx;
  const double* __restrict__ w = a.tab.w;
  const double* __restrict__ Phi = a.tab.Phi;
  const int MQ = M * Q;
  double* s_part = s_v + MQ;
  // projection split: warp k sums the nodes [k qw, (k+1) qw) for every entry, lanes over entries
  const int qw = (Q + UWARPS - 1) / UWARPS;
  const int q_lo = min(Q, warp * qw), q_hi = min(Q, q_lo + qw);

  for (int j = blockIdx.x + 1; j <= a.nx; j += gridDim.x) {
    const int jl = neighbour(j, a.nx, -1, a.bc_left);
    const int jr = neighbour(j, a.nx, +1, a.bc_right);
    const double* ul_g = a.unode + (size_t)jl * MQ;
    const double* uc_g = a.unode + (size_t)j * MQ;
    const double* ur_g = a.unode + (size_t)jr * MQ;
    for (int q = tid; q < Q; q += UT) {
      double ul[M], uc[M], ur[M], fl[M], fc[M], fr[M];
#pragma unroll
      for (int c = 0; c < M; ++c) {
        ul[c] = ul_g[c * Q + q];
        uc[c] = uc_g[c * Q + q];
        ur[c] = ur_g[c * Q + q];
      }
      Flux1D<PHYS, M>::f(ul, a.gamma, fl);
      Flux1D<PHYS, M>::f(uc, a.gamma, fc);
      Flux1D<PHYS, M>::f(ur, a.gamma, fr);
      const double wq = w[q];
#pragma unroll
      for (int c = 0; c < M; ++c) {
        const double gR = 0.5 * (fc[c] + fr[c]) - nu * (ur[c] - uc[c]);
        const double gL = 0.5 * (fl[c] + fc[c]) - nu * (uc[c] - ul[c]);
        s_v[c * Q + q] = wq * (uc[c] - r * (gR - gL));
      }
    }
    __syncthreads();
    double* out = a.uhat + (size_t)j * NM;
    const double old00 = out[0];
    __syncthreads();                                       // everyone read the old value before it changes
    // ghost targets that mirror this cell
    const int g0 = (j == 1 && a.bc_left == IPM_BC_OUTFLOW) || (j == a.nx && a.bc_left == IPM_BC_PERIODIC);
    const int g1 = (j == a.nx && a.bc_right == IPM_BC_OUTFLOW) || (j == 1 && a.bc_right == IPM_BC_PERIODIC);
    double* out0 = a.uhat;                                 // ghost 0
    double* out1 = a.uhat + (size_t)(a.nx + 1) * NM;       // ghost nx+1
    // projection u_hat_(i,c) = sum_q phi_i(xi_q) v_c(xi_q): partial sums per warp, added in warp order
    for (int rr = lane; rr < NM; rr += 32) {
      const int i = rr / M, c = rr - i * M;
      double acc = 0.0;
      for (int q = q_lo; q < q_hi; ++q) acc = fma(Phi[(size_t)q * N + i], s_v[c * Q + q], acc);
      s_part[warp * NM + rr] = acc;
    }
    __syncthreads();
    for (int rr = tid; rr < NM; rr += UT) {
      double v = 0.0;
#pragma unroll
      for (int k = 0; k < UWARPS; ++k) v += s_part[k * NM + rr];
      out[rr] = v;
      if (g0) out0[rr] = v;
      if (g1) out1[rr] = v;
    }
    if (g0 || g1) {
      const double* lj = a.lam + (size_t)j * NM;
      for (int rr = tid; rr < NM; rr += UT) {
        const double v = lj[rr];
        if (g0) a.lam[rr] = v;
        if (g1) a.lam[(size_t)(a.nx + 1) * NM + rr] = v;
      }
    }
    __syncthreads();
    if (tid == 0 && a.cell_resid) a.cell_resid[j] = a.dx * fabs(out[0] - old00);
    __syncthreads();
  }
}

// The Lax-Friedrichs update from the terms the Newton launch folded (lf_fold in newton.cu):
// u_hat_j = A_j - (dt/dx) B_j, with dt from the speeds of this solve; ghost copies and the steady
// residual as in k_update1d.
__global__ void __launch_bounds__(UT) k_lf_combine(Update1DArgs a, int NM, const double* __restrict__ lf_a,
                                                   const double* __restrict__ lf_b) {
  const int tid = threadIdx.x;
  const double dt = step_dt(a);
  if (blockIdx.x == 0 && tid == 0) a.sc->dt = dt > 0.0 ? dt : 0.0;
  if (!(dt > 0.0)) return;
  const double r = dt / a.dx;
  for (int j = blockIdx.x + 1; j <= a.nx; j += gridDim.x) {
    double* out = a.uhat + (size_t)j * NM;
    const double old00 = out[0];                       // thread 0 reads it before it writes entry 0
    const int g0 = (j == 1 && a.bc_left == IPM_BC_OUTFLOW) || (j == a.nx && a.bc_left == IPM_BC_PERIODIC);
    const int g1 = (j == a.nx && a.bc_right == IPM_BC_OUTFLOW) || (j == 1 && a.bc_right == IPM_BC_PERIODIC);
    double* out0 = a.uhat;
    double* out1 = a.uhat + (size_t)(a.nx + 1) * NM;
    const double* A = lf_a + (size_t)j * NM;
    const double* B = lf_b + (size_t)j * NM;
    for (int rr = tid; rr < NM; rr += UT) {
      const double v = fma(-r, B[rr], A[rr]);
      if (rr == 0 && a.cell_resid) a.cell_resid[j] = a.dx * fabs(v - old00);
      out[rr] = v;
      if (g0) out0[rr] = v;
      if (g1) out1[rr] = v;
    }
    if (g0 || g1) {
      const double* lj = a.lam + (size_t)j * NM;
      for (int rr = tid; rr < NM; rr += UT) {
        const double v = lj[rr];
        if (g0) a.lam[rr] = v;
        if (g1) a.lam[(size_t)(a.nx + 1) * NM + rr] = v;
      }
    }
  }
}

cudaError_t launch_lf_combine(const Update1DArgs& a, int NM, const double* lf_a, const double* lf_b, int grid,
                              cudaStream_t s) {
  k_lf_combine<<<grid, UT, 0, s>>>(a, NM, lf_a, lf_b);
  return cudaGetLastError();
}

static size_t update1d_smem(int m, int N, int Q) { return ((size_t)m * Q + (size_t)UWARPS * N * m) * sizeof(double); }

cudaError_t prepare_update1d(int phys, int m, int N, int Q) {
  const size_t smem = update1d_smem(m, N, Q);
  if (phys == PHYS_BURGERS && m == 1) return raise_smem_limit(k_update1d<PHYS_BURGERS, 1>, smem);
  if (phys == PHYS_EULER1D && m == 3) return raise_smem_limit(k_update1d<PHYS_EULER1D, 3>, smem);
  return cudaErrorInvalidValue;
}

cudaError_t launch_update1d(int phys, int m, const Update1DArgs& a, int grid, cudaStream_t s) {
  const size_t smem = update1d_smem(m, a.tab.N, a.tab.Q);
  if (phys == PHYS_BURGERS && m == 1) {
    k_update1d<PHYS_BURGERS, 1><<<grid, UT, smem, s>>>(a);
  } else if (phys == PHYS_EULER1D && m == 3) {
    k_update1d<PHYS_EULER1D, 3><<<grid, UT, smem, s>>>(a);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Initial data (Algorithm 1, first loop): exact nodal cell averages of the Riemann data, projected;
// initial duals = projection of grad s of the nodal averages.
// ------------------------------------------------------------------------------------------------
struct InitArgs {
  Tables tab;
  EntParams ent;
  IC1D ic;
  double* uhat;
  double* lam;
  int n_cells;
};

template <int ENT, int M>
__global__ void __launch_bounds__(UT) k_init1d(InitArgs a) {
  extern __shared__ __align__(16) double sm[];
  const int N = a.tab.N, Q = a.tab.Q, P = a.tab.p, NM = N * M;
  double* s_u = sm;            // [M][Q] w * ubar
  double* s_e = sm + M * Q;    // [M][Q] w * grad s(ubar)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int j = blockIdx.x; j < a.n_cells; j += gridDim.x) {
    for (int q = tid; q < Q; q += UT) {
      double xi[3] = {0.0, 0.0, 0.0};
      for (int d = 0; d < P; ++d) xi[d] = a.tab.nodes[(size_t)q * P + d];
      double ub[M], ge[M];
      ic1d_average<M>(a.ic, j, xi, P, ub);
      entropy_gradient<ENT, M>(ub, a.ent, ge);
      const double wq = a.tab.w[q];
#pragma unroll
      for (int c = 0; c < M; ++c) {
        s_u[c * Q + q] = wq * ub[c];
        s_e[c * Q + q] = wq * ge[c];
      }
    }
    __syncthreads();
    for (int i = warp; i < N; i += UWARPS) {
      double au[M], ae[M];
#pragma unroll
      for (int c = 0; c < M; ++c) au[c] = ae[c] = 0.0;
      for (int q = lane; q < Q; q += 32) {
        const double ph = a.tab.PhiT[(size_t)i * Q + q];
#pragma unroll
        for (int c = 0; c < M; ++c) {
          au[c] = fma(ph, s_u[c * Q + q], au[c]);
          ae[c] = fma(ph, s_e[c * Q + q], ae[c]);
        }
      }
#pragma unroll
      for (int c = 0; c < M; ++c) {
        const double vu = warp_sum(au[c]), ve = warp_sum(ae[c]);
        if (lane == 0) {
          a.uhat[(size_t)j * NM + i * M + c] = vu;
          a.lam[(size_t)j * NM + i * M + c] = ve;
        }
      }
    }
    __syncthreads();
  }
}

cudaError_t launch_init1d(int ent, int m, const Tables& tab, const EntParams& ent_p, const ipm_problem& prob,
                          double* uhat, double* lam, int n_cells, cudaStream_t s) {
  InitArgs a;
  a.tab = tab;
  a.ent = ent_p;
  a.ic = ic1d_params(prob);
  a.uhat = uhat;
  a.lam = lam;
  a.n_cells = n_cells;
  const size_t smem = 2 * (size_t)m * tab.Q * sizeof(double);
  const int grid = n_cells < 4096 ? n_cells : 4096;
#define IPM_INIT_CASE(E, MM)                                                                              \
  if (ent == E && m == MM) {                                                                              \
    if (smem > 48 * 1024) {                                                                               \
      const cudaError_t e_ = raise_smem_limit(k_init1d<E, MM>, smem);                                     \
      if (e_ != cudaSuccess) return e_;                                                                   \
    }                                                                                                     \
    k_init1d<E, MM><<<grid, UT, smem, s>>>(a);                                                            \
    return cudaGetLastError();                                                                            \
  }
  IPM_INIT_CASE(ENT_BARRIER, 1)
  IPM_INIT_CASE(ENT_QUADRATIC, 1)
  IPM_INIT_CASE(ENT_EULER, 3)
  IPM_INIT_CASE(ENT_QUADRATIC, 3)
#undef IPM_INIT_CASE
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------------------------------------
// Boundary copies of moments and duals (outflow / periodic ghosts).
// ------------------------------------------------------------------------------------------------
__global__ void k_bc_copy1d(double* uhat, double* lam, int nx, int Nm, int bcl, int bcr) {
  for (int r = threadIdx.x; r < Nm; r += blockDim.x) {
    if (bcl != IPM_BC_DIRICHLET) {
      const int src = bcl == IPM_BC_OUTFLOW ? 1 : nx;
      uhat[r] = uhat[(size_t)src * Nm + r];
      lam[r] = lam[(size_t)src * Nm + r];
    }
    if (bcr != IPM_BC_DIRICHLET) {
      const int src = bcr == IPM_BC_OUTFLOW ? nx : 1;
      uhat[(size_t)(nx + 1) * Nm + r] = uhat[(size_t)src * Nm + r];
      lam[(size_t)(nx + 1) * Nm + r] = lam[(size_t)src * Nm + r];
    }
  }
}

cudaError_t launch_bc_copy1d(double* uhat, double* lam, int nx, int Nm, int bcl, int bcr, cudaStream_t s) {
  k_bc_copy1d<<<1, 256, 0, s>>>(uhat, lam, nx, Nm, bcl, bcr);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Per-step bookkeeping: advance t, reduce per-cell counters and the residual in a fixed order,
// reset the queue counter and the speed maximum for the next launch.
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_finalize(StepScalars* sc, const int* iters, const int* status,
                                                  const double* cell_resid, int first, int count, int advance) {
  __shared__ double s_res[256];
  __shared__ long long s_it[256];
  __shared__ int s_max[256], s_fail[256], s_first[256];
  const int tid = threadIdx.x;
  double res = 0.0;
  long long itsum = 0;
  int imax = 0, nfail = 0, ffirst = 0x7fffffff;
  // contiguous chunk per thread: fixed summation order
  const int chunk = (count + 255) / 256;
  const int lo = first + tid * chunk, hi = min(first + count, lo + chunk);
  for (int c = lo; c < hi; ++c) {
    if (cell_resid) res += cell_resid[c];
    itsum += iters[c];
    imax = max(imax, iters[c]);
    if (status[c] != 0) {
      ++nfail;
      ffirst = min(ffirst, c);
    }
  }
  s_res[tid] = res;
  s_it[tid] = itsum;
  s_max[tid] = imax;
  s_fail[tid] = nfail;
  s_first[tid] = ffirst;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (tid < o) {
      s_res[tid] += s_res[tid + o];
      s_it[tid] += s_it[tid + o];
      s_max[tid] = max(s_max[tid], s_max[tid + o]);
      s_fail[tid] += s_fail[tid + o];
      s_first[tid] = min(s_first[tid], s_first[tid + o]);
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (advance && sc->dt > 0.0) {
      sc->t += sc->dt;
      sc->steps += 1;
    }
    sc->residual = s_res[0];
    sc->newton_iters = s_it[0];
    sc->max_iters = s_max[0];
    sc->failed_cells = s_fail[0];
    sc->first_failed_cell = s_fail[0] ? s_first[0] : -1;
    sc->first_status = s_fail[0] ? status[s_first[0]] : 0;
    sc->last_factorizations = sc->factorizations;
    sc->factorizations = 0;
    sc->last_cached_checks = sc->cached_checks;
    sc->cached_checks = 0;
    sc->last_hessian_ns = sc->hessian_ns;
    sc->hessian_ns = 0;
    sc->last_hessian_count = sc->hessian_count;
    sc->hessian_count = 0;
    sc->work_counter = 0;
    sc->update_counter = 0;
    sc->smax_bits = sc->fixed_smax_bits;
  }
}

cudaError_t launch_finalize(StepScalars* sc, const int* iters, const int* status, const double* cell_resid,
                            int n_cells, int first, int count, int advance_time, cudaStream_t s) {
  (void)n_cells;
  k_finalize<<<1, 256, 0, s>>>(sc, iters, status, cell_resid, first, count, advance_time);
  return cudaGetLastError();
}

}  // namespace ipm
