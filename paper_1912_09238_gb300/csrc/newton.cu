// newton.cu -- per-cell Newton solve of the IPM dual problem, FP64 path.
//
// One CTA owns one cell at a time and pulls cells from a persistent work queue (an atomic
// counter bounded by the number of cells), so cells with uneven Newton counts balance out.
// Per Newton iteration, all on chip (Sec. 3.1):
//   (a1) Lambda_k = sum_i lambda_i phi_i(xi_k)                           reconstruction
//   (a2) u_k = u_s(Lambda_k), J_k = grad u_s(Lambda_k), s_*(Lambda_k)     closure per node
//   (a3) grad L = sum_k w_k u_k phi(xi_k)^T - u_hat; stop if Eq. tauCrit holds
//   (b)  H((i,a),(j,b)) = sum_k w_k J_k,ab phi_i(xi_k) phi_j(xi_k)        packed lower triangle
//   (c)  H = L L^T (right-looking Cholesky), Delta = -H^-1 grad L (one warp), then Armijo
//        backtracking on L (Eq. L) along Delta using Lambda + alpha Phi Delta.
// The packed Hessian lives in shared memory when it fits, else in a per-CTA slot of a global
// workspace (L2-resident).
//
// Every loop is bounded: the queue by the cell count, Newton by max_newton, the line search by
// max_halvings, the factorisation and solves by N*m.
#include <type_traits>

#include "ipm_host.h"

namespace ipm {

constexpr int NT = 256;
constexpr int NWARPS = NT / 32;

template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* s_red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) s_red[warp * K + k] = v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = 0.0;
    for (int w = 0; w < NWARPS; ++w) s += s_red[w * K + k];
    v[k] = s;
  }
  __syncthreads();
}

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

template <int ENT, int PHYS, int M, bool H_SMEM>
__global__ void __launch_bounds__(NT) k_newton(NewtonArgs a) {
  constexpr int B = packed_count(M);
  extern __shared__ __align__(16) double smem[];
  __shared__ int s_work;
  const int N = a.tab.N, Q = a.tab.Q, NM = N * M;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double* s_lam = smem;
  double* s_uh = s_lam + NM;
  double* s_g = s_uh + NM;
  double* s_d = s_g + NM;
  double* s_Lam = s_d + NM;       // [M][Q]
  double* s_dLam = s_Lam + M * Q; // [M][Q]
  double* s_u = s_dLam + M * Q;   // [M][Q]
  double* s_wJ = s_u + M * Q;     // [B][Q]
  double* s_red = s_wJ + B * Q;   // NWARPS * 8
  double* s_H = H_SMEM ? (s_red + NWARPS * 8) : (a.hwork + (size_t)blockIdx.x * a.hwork_stride);
  const double* __restrict__ PhiT = a.tab.PhiT;
  const double* __restrict__ Phi = a.tab.Phi;
  const double* __restrict__ w = a.tab.w;
  const uint32_t* __restrict__ pairs = a.tab.pairs;
  const int NP = N * (N + 1) / 2;

  for (;;) {
    if (tid == 0) s_work = atomicAdd(&a.sc->work_counter, 1);
    __syncthreads();
    const int wk = s_work;
    if (wk >= a.n_work) break;
    const int cell = a.cell_list ? a.cell_list[wk] : (wk / a.nx + a.gy) * (a.nx + 2) + (wk % a.nx + 1);
    double* lam_g = a.lam + (size_t)cell * NM;
    const double* uh_g = a.uhat + (size_t)cell * NM;
    for (int r = tid; r < NM; r += NT) {
      s_lam[r] = lam_g[r];
      s_uh[r] = uh_g[r];
    }
    __syncthreads();

    int it = 0, st = ST_OK;
    for (;;) {
      // (a1) reconstruction
      for (int q = tid; q < Q; q += NT) {
        double acc[M];
#pragma unroll
        for (int c = 0; c < M; ++c) acc[c] = 0.0;
        for (int i = 0; i < N; ++i) {
          const double ph = PhiT[(size_t)i * Q + q];
#pragma unroll
          for (int c = 0; c < M; ++c) acc[c] = fma(ph, s_lam[i * M + c], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < M; ++c) s_Lam[c * Q + q] = acc[c];
      }
      __syncthreads();
      // (a2) closure, cost terms
      double red[5] = {0.0, 0.0, 0.0, 0.0, 0.0};  // sum w s*, sum w |s*|, #infeasible, lambda.uhat, sum |lambda uhat|
      for (int q = tid; q < Q; q += NT) {
        double L[M], u[M], J[B], ss;
#pragma unroll
        for (int c = 0; c < M; ++c) L[c] = s_Lam[c * Q + q];
        const bool ok = Closure<ENT, M>::template eval<true>(L, a.ent, u, J, ss);
        const double wq = w[q];
#pragma unroll
        for (int c = 0; c < M; ++c) s_u[c * Q + q] = u[c];
#pragma unroll
        for (int b = 0; b < B; ++b) s_wJ[b * Q + q] = wq * J[b];
        red[0] = fma(wq, ss, red[0]);
        red[1] = fma(wq, fabs(ss), red[1]);
        red[2] += ok ? 0.0 : 1.0;
      }
      for (int r = tid; r < NM; r += NT) {
        const double t = s_lam[r] * s_uh[r];
        red[3] += t;
        red[4] += fabs(t);
      }
      block_sum<5>(red, s_red);
      const double L0 = red[0] - red[3];
      const double slack = a.slack_rel * (1.0 + red[1] + red[4]);
      // (a3) gradient, one warp per moment
      double gpart = 0.0;
      for (int i = warp; i < N; i += NWARPS) {
        double acc[M];
#pragma unroll
        for (int c = 0; c < M; ++c) acc[c] = 0.0;
        for (int q = lane; q < Q; q += 32) {
          const double ph = w[q] * PhiT[(size_t)i * Q + q];
#pragma unroll
          for (int c = 0; c < M; ++c) acc[c] = fma(ph, s_u[c * Q + q], acc[c]);
        }
        double nrm = 0.0;
#pragma unroll
        for (int c = 0; c < M; ++c) {
          const double gi = warp_sum(acc[c]) - s_uh[i * M + c];
          nrm = fma(gi, gi, nrm);
          if (lane == 0) s_g[i * M + c] = gi;
        }
        gpart += sqrt(nrm);
      }
      if (lane == 0) s_red[warp] = gpart;
      __syncthreads();
      double res = 0.0;
      for (int ww = 0; ww < NWARPS; ++ww) res += s_red[ww];
      __syncthreads();

      if (red[2] > 0.0) { st = ST_INFEASIBLE; break; }
      if (!isfinite(res)) { st = ST_NONFINITE; break; }
      if (a.one_step) {
        if (it >= 1) break;
      } else {
        if (res < a.tau) break;
        if (it >= a.max_newton) { st = ST_NOCONV; break; }
      }

      // (b) Hessian, packed lower triangle, row index r = i*M + a
      for (int pidx = tid; pidx < NP; pidx += NT) {
        const uint32_t pr = pairs[pidx];
        const int i = (int)(pr >> 16), j = (int)(pr & 0xffffu);
        double acc[B];
#pragma unroll
        for (int b = 0; b < B; ++b) acc[b] = 0.0;
        for (int q = 0; q < Q; ++q) {
          const double pq = Phi[(size_t)q * N + i] * Phi[(size_t)q * N + j];
#pragma unroll
          for (int b = 0; b < B; ++b) acc[b] = fma(s_wJ[b * Q + q], pq, acc[b]);
        }
#pragma unroll
        for (int a1 = 0; a1 < M; ++a1)
#pragma unroll
          for (int b1 = 0; b1 < M; ++b1) {
            const int r = i * M + a1, c = j * M + b1;
            if (r < c) continue;
            const int lo = a1 < b1 ? a1 : b1, hi = a1 < b1 ? b1 : a1;
            s_H[(size_t)r * (r + 1) / 2 + c] = acc[packed_ab(lo, hi, M)];
          }
      }
      __syncthreads();

      // (c) Cholesky in place
      bool spd = true;
      for (int k = 0; k < NM; ++k) {
        const size_t kk = (size_t)k * (k + 1) / 2 + k;
        const double dkk = s_H[kk];
        if (!(dkk > 0.0) || !isfinite(dkk)) { spd = false; break; }
        const double d = sqrt(dkk), id = 1.0 / d;
        for (int i = k + 1 + tid; i < NM; i += NT) s_H[(size_t)i * (i + 1) / 2 + k] *= id;
        __syncthreads();
        if (tid == 0) s_H[kk] = d;
        for (int i = k + 1 + warp; i < NM; i += NWARPS) {
          const size_t ri = (size_t)i * (i + 1) / 2;
          const double lik = s_H[ri + k];
          for (int j = k + 1 + lane; j <= i; j += 32) s_H[ri + j] = fma(-lik, s_H[(size_t)j * (j + 1) / 2 + k], s_H[ri + j]);
        }
        __syncthreads();
      }
      if (!spd) { st = ST_NOTSPD; break; }
      // triangular solves with one warp: L y = -g, L^T Delta = y
      if (warp == 0) {
        for (int r = lane; r < NM; r += 32) s_d[r] = -s_g[r];
        __syncwarp();
        for (int k = 0; k < NM; ++k) {
          const double yk = s_d[k] / s_H[(size_t)k * (k + 1) / 2 + k];
          __syncwarp();
          for (int i = k + 1 + lane; i < NM; i += 32) s_d[i] = fma(-s_H[(size_t)i * (i + 1) / 2 + k], yk, s_d[i]);
          if (lane == 0) s_d[k] = yk;
          __syncwarp();
        }
        for (int k = NM - 1; k >= 0; --k) {
          const size_t rk = (size_t)k * (k + 1) / 2;
          const double xk = s_d[k] / s_H[rk + k];
          __syncwarp();
          for (int i = lane; i < k; i += 32) s_d[i] = fma(-s_H[rk + i], xk, s_d[i]);
          if (lane == 0) s_d[k] = xk;
          __syncwarp();
        }
      }
      __syncthreads();
      // direction at the nodes, slope, Delta . u_hat
      for (int q = tid; q < Q; q += NT) {
        double acc[M];
#pragma unroll
        for (int c = 0; c < M; ++c) acc[c] = 0.0;
        for (int i = 0; i < N; ++i) {
          const double ph = PhiT[(size_t)i * Q + q];
#pragma unroll
          for (int c = 0; c < M; ++c) acc[c] = fma(ph, s_d[i * M + c], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < M; ++c) s_dLam[c * Q + q] = acc[c];
      }
      double r2[2] = {0.0, 0.0};
      for (int r = tid; r < NM; r += NT) {
        r2[0] = fma(s_g[r], s_d[r], r2[0]);
        r2[1] = fma(s_d[r], s_uh[r], r2[1]);
      }
      block_sum<2>(r2, s_red);
      const double slope = r2[0], dU = r2[1];
      // Armijo backtracking
      double alpha = 1.0;
      bool accepted = false;
      for (int h = 0; h <= a.max_halvings; ++h) {
        double rr[2] = {0.0, 0.0};
        for (int q = tid; q < Q; q += NT) {
          double L[M], ss;
#pragma unroll
          for (int c = 0; c < M; ++c) L[c] = fma(alpha, s_dLam[c * Q + q], s_Lam[c * Q + q]);
          const bool ok = Closure<ENT, M>::feasible_sstar(L, a.ent, ss);
          rr[0] = fma(w[q], ss, rr[0]);
          rr[1] += ok ? 0.0 : 1.0;
        }
        block_sum<2>(rr, s_red);
        const double Lt = rr[0] - fma(alpha, dU, red[3]);
        if (rr[1] == 0.0 && isfinite(Lt) && Lt <= L0 + a.armijo_c * alpha * slope + slack) {
          accepted = true;
          break;
        }
        alpha *= 0.5;
      }
      if (!accepted) { st = ST_LINESEARCH; break; }
      for (int r = tid; r < NM; r += NT) s_lam[r] = fma(alpha, s_d[r], s_lam[r]);
      __syncthreads();
      ++it;
    }

    // results: duals, nodal states at the final duals, counters, signal speed
    for (int r = tid; r < NM; r += NT) lam_g[r] = s_lam[r];
    double* un = a.unode + (size_t)cell * M * Q;
    for (int r = tid; r < M * Q; r += NT) un[r] = s_u[r];
    if (tid == 0) {
      a.iters[cell] = it;
      a.status[cell] = st;
    }
    if (a.track_speed) {
      double smax = 0.0;
      for (int q = tid; q < Q; q += NT) {
        double u[M];
#pragma unroll
        for (int c = 0; c < M; ++c) u[c] = s_u[c * Q + q];
        smax = fmax(smax, node_speed<PHYS, M>(u, a.ent.gamma));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
      if (lane == 0) s_red[warp] = smax;
      __syncthreads();
      if (tid == 0) {
        double v = 0.0;
        for (int ww = 0; ww < NWARPS; ++ww) v = fmax(v, s_red[ww]);
        atomic_max_pos(&a.sc->smax_bits, v);
      }
    }
    __syncthreads();
  }
}

int newton_threads() { return NT; }

size_t newton_smem_bytes(int N, int m, int Q, bool h_in_smem) {
  const size_t NM = (size_t)N * m;
  const size_t B = (size_t)m * (m + 1) / 2;
  size_t d = 4 * NM + 3 * (size_t)m * Q + B * Q + NWARPS * 8;
  if (h_in_smem) d += NM * (NM + 1) / 2;
  return d * sizeof(double);
}

// prepare = 1: raise the kernel's dynamic shared-memory limit (outside any stream capture);
// prepare = 0: launch.
template <int ENT, int PHYS, int M>
static cudaError_t launch_t(const NewtonArgs* a, int grid, size_t smem, bool h_in_smem, cudaStream_t s, int prepare,
                            int* blocks_per_sm) {
  auto k = h_in_smem ? k_newton<ENT, PHYS, M, true> : k_newton<ENT, PHYS, M, false>;
  if (prepare) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, NT, smem);
  }
  k<<<grid, NT, smem, s>>>(*a);
  return cudaGetLastError();
}

template <typename F>
static cudaError_t dispatch(int ent, int phys, int m, F&& f) {
  if (phys == PHYS_BURGERS && m == 1) {
    if (ent == ENT_BARRIER) return f(std::integral_constant<int, ENT_BARRIER>(), std::integral_constant<int, PHYS_BURGERS>(), std::integral_constant<int, 1>());
    if (ent == ENT_QUADRATIC) return f(std::integral_constant<int, ENT_QUADRATIC>(), std::integral_constant<int, PHYS_BURGERS>(), std::integral_constant<int, 1>());
  }
  if (phys == PHYS_EULER1D && m == 3) {
    if (ent == ENT_EULER) return f(std::integral_constant<int, ENT_EULER>(), std::integral_constant<int, PHYS_EULER1D>(), std::integral_constant<int, 3>());
    if (ent == ENT_QUADRATIC) return f(std::integral_constant<int, ENT_QUADRATIC>(), std::integral_constant<int, PHYS_EULER1D>(), std::integral_constant<int, 3>());
  }
  if (phys == PHYS_EULER2D && m == 4) {
    if (ent == ENT_EULER) return f(std::integral_constant<int, ENT_EULER>(), std::integral_constant<int, PHYS_EULER2D>(), std::integral_constant<int, 4>());
    if (ent == ENT_QUADRATIC) return f(std::integral_constant<int, ENT_QUADRATIC>(), std::integral_constant<int, PHYS_EULER2D>(), std::integral_constant<int, 4>());
  }
  return cudaErrorInvalidValue;
}

cudaError_t prepare_newton(int ent, int phys, int m, size_t smem, bool h_in_smem, int* blocks_per_sm) {
  return dispatch(ent, phys, m, [&](auto E, auto P, auto MM) {
    return launch_t<decltype(E)::value, decltype(P)::value, decltype(MM)::value>(nullptr, 0, smem, h_in_smem, nullptr, 1,
                                                                                   blocks_per_sm);
  });
}

// phys is the PhysKind; ent the EntKind.
cudaError_t launch_newton_phys(int ent, int phys, int m, const NewtonArgs& a, int grid, size_t smem, bool h_in_smem,
                               cudaStream_t s) {
  return dispatch(ent, phys, m, [&](auto E, auto P, auto MM) {
    return launch_t<decltype(E)::value, decltype(P)::value, decltype(MM)::value>(&a, grid, smem, h_in_smem, s, 0,
                                                                                   nullptr);
  });
}

}  // namespace ipm
