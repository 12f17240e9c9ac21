// newton_warp.cu -- the per-cell Newton solve of the IPM dual problem for small cells (N*m <= 64):
// one warp per cell, several warps (cells) per CTA.
//
// The steps are those of newton.cu (Sec. 3.1: reconstruction, closure, gradient and Eq. tauCrit,
// Hessian, Cholesky with the gradient as augmented row, back substitution, Armijo line search on
// Eq. L), but every reduction is a warp shuffle and every barrier a __syncwarp, so the many small
// cells of a mesh proceed independently: a 256-thread CTA per cell would spend most of its time
// in block-wide barriers for matrices of 6 to 64 rows. Each warp pulls its own cells from the
// persistent queue.
//
// Precision. FP64 path: all in float64. Mixed path: the Hessian entries are FP32 products
// accumulated in FP32 (w_k J_k,ab rounded to FP32 times phi_i phi_j in FP32) on the CUDA cores --
// a tensor-core tile of 128 rows is not filled by one small cell -- and widened to float64; the
// gradient, stopping test, factorisation, solves and line search stay float64.
//
// Every loop is bounded as in newton.cu (queue, max_newton, max_halvings, N*m).
#include <type_traits>

#include "ipm_host.h"

namespace ipm {

__device__ __forceinline__ size_t rowoff_w(int r) { return (size_t)r * (r + 1) / 2; }
__device__ __forceinline__ int work_cell_w(int w, int nx, int gy) { return (w / nx + gy) * (nx + 2) + (w % nx + 1); }

template <int K>
__device__ __forceinline__ void warp_sums(double (&v)[K]) {
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
}

// doubles of one warp's shared-memory slice
__host__ __device__ inline size_t warp_slice_doubles(int N, int m, int Q) {
  const size_t NM = (size_t)N * m, B = (size_t)m * (m + 1) / 2;
  return 5 * NM + 4 * (size_t)m * Q + B * Q + (NM + 1) * (NM + 2) / 2;
}

// The 1-D Lax-Friedrichs update folded into the launch, one warp (as lf_fold in newton.cu): once the
// nodal states of cell k are final, count k towards each cell it neighbours; for each count this warp
// completes, form that cell's A = P(w (u_l + u_r)/2) and B = P(w (f(u_r) - f(u_l))/2), lanes over the
// nodes for the integrands and over the entries for the projections. Scratch s_ia, s_ib [M][Q].
template <int PHYS, int M>
__device__ void lf_fold_warp(const NewtonArgs& a, int k, double* s_ia, double* s_ib) {
  const int lane = threadIdx.x & 31;
  const int nx = a.nx, Q = a.tab.Q, N = a.tab.N, NM = N * M;
  __threadfence();                                   // this warp's nodal states of k, before the counts
  __syncwarp();
  int n = 0, r0 = 0, r1 = 0, r2 = 0;
  if (lane == 0) {
    const int cand[5] = {k - 1, k + 1, k, 1, nx};
    for (int ci = 0; ci < 5; ++ci) {
      const int j = cand[ci];
      bool seen = j < 1 || j > nx;
      for (int cj = 0; cj < ci; ++cj) seen = seen || cand[cj] == j;
      if (seen) continue;
      const int jl = neighbour(j, nx, -1, a.bc_left), jr = neighbour(j, nx, +1, a.bc_right);
      const bool il = jl >= 1 && jl <= nx, ir = jr >= 1 && jr <= nx && jr != jl;
      const int target = (il ? 1 : 0) + (ir ? 1 : 0);
      bool ready = false;
      if (target == 0) ready = j == k;
      else if (jl == k || jr == k) ready = atomicAdd(&a.lf_cnt[j], 1) == target - 1;
      if (ready) {
        if (n == 0) r0 = j;
        else if (n == 1) r1 = j;
        else r2 = j;
        ++n;
      }
    }
    __threadfence();                                 // the other warps' nodal states, after the counts
  }
  n = __shfl_sync(0xffffffffu, n, 0);
  r0 = __shfl_sync(0xffffffffu, r0, 0);
  r1 = __shfl_sync(0xffffffffu, r1, 0);
  r2 = __shfl_sync(0xffffffffu, r2, 0);
  const double* __restrict__ w = a.tab.w;
  const double* __restrict__ Phi = a.tab.Phi;
  for (int t = 0; t < n; ++t) {
    const int j = t == 0 ? r0 : (t == 1 ? r1 : r2);
    const double* ul_g = a.unode + (size_t)neighbour(j, nx, -1, a.bc_left) * M * Q;
    const double* ur_g = a.unode + (size_t)neighbour(j, nx, +1, a.bc_right) * M * Q;
    for (int q = lane; q < Q; q += 32) {
      double ul[M], ur[M], fl[M], fr[M];
#pragma unroll
      for (int c = 0; c < M; ++c) {
        ul[c] = ul_g[c * Q + q];
        ur[c] = ur_g[c * Q + q];
      }
      Flux1D<PHYS, M>::f(ul, a.ent.gamma, fl);
      Flux1D<PHYS, M>::f(ur, a.ent.gamma, fr);
      const double wq = w[q];
#pragma unroll
      for (int c = 0; c < M; ++c) {
        s_ia[c * Q + q] = wq * (0.5 * (ul[c] + ur[c]));
        s_ib[c * Q + q] = wq * (0.5 * (fr[c] - fl[c]));
      }
    }
    __syncwarp();
    for (int rr = lane; rr < NM; rr += 32) {
      const int i = rr / M, c = rr - i * M;
      double sa = 0.0, sb = 0.0;
      for (int q = 0; q < Q; ++q) {
        const double ph = Phi[(size_t)q * N + i];
        sa = fma(ph, s_ia[c * Q + q], sa);
        sb = fma(ph, s_ib[c * Q + q], sb);
      }
      a.lf_a[(size_t)j * NM + rr] = sa;
      a.lf_b[(size_t)j * NM + rr] = sb;
    }
    __syncwarp();
  }
}

template <int ENT, int PHYS, int M, bool MIXED>
__global__ void __launch_bounds__(256) k_newton_warp(NewtonArgs a, int slice) {
  constexpr int B = packed_count(M);
  extern __shared__ __align__(16) double wsm[];
  const int N = a.tab.N, Q = a.tab.Q, NM = N * M;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* base = wsm + (size_t)warp * slice;
  double* s_lam = base;
  double* s_uh = s_lam + NM;
  double* s_g = s_uh + NM;
  double* s_d = s_g + NM;
  double* s_dinv = s_d + NM;
  double* s_Lam = s_dinv + NM;    // [M][Q]
  double* s_dLam = s_Lam + M * Q; // [M][Q]
  double* s_u = s_dLam + M * Q;   // [M][Q]
  double* s_wu = s_u + M * Q;     // [M][Q]
  double* s_wJ = s_wu + M * Q;    // [B][Q] (float on the mixed path)
  double* s_H = s_wJ + B * Q;     // packed (NM+1)(NM+2)/2
  const double* __restrict__ PhiT = a.tab.PhiT;
  const double* __restrict__ Phi = a.tab.Phi;
  const double* __restrict__ w = a.tab.w;
  const int NP = N * (N + 1) / 2;

  for (;;) {
    int wk = 0;
    if (lane == 0) wk = atomicAdd(&a.sc->work_counter, 1);
    wk = __shfl_sync(0xffffffffu, wk, 0);
    if (wk >= a.n_work) break;
    const int cell = a.cell_list ? a.cell_list[wk] : work_cell_w(wk, a.nx, a.gy);
    double* lam_g = a.lam + (size_t)cell * NM;
    const double* uh_g = a.uhat + (size_t)cell * NM;
    for (int r = lane; r < NM; r += 32) {
      s_lam[r] = lam_g[r];
      s_uh[r] = uh_g[r];
    }
    __syncwarp();
    int it = 0, st = ST_OK;
    for (;;) {
      // (a1) reconstruction, (a2) closure and cost terms, lanes over nodes
      double red[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
      for (int q = lane; q < Q; q += 32) {
        double L[M], u[M], J[B], ss;
#pragma unroll
        for (int c = 0; c < M; ++c) L[c] = 0.0;
        for (int i = 0; i < N; ++i) {
          const double ph = PhiT[(size_t)i * Q + q];
#pragma unroll
          for (int c = 0; c < M; ++c) L[c] = fma(ph, s_lam[i * M + c], L[c]);
        }
        const bool ok = Closure<ENT, M>::template eval<true>(L, a.ent, u, J, ss);
        const double wq = w[q];
#pragma unroll
        for (int c = 0; c < M; ++c) {
          s_Lam[c * Q + q] = L[c];
          s_u[c * Q + q] = u[c];
          s_wu[c * Q + q] = wq * u[c];
        }
        if (MIXED) {
          float* f = reinterpret_cast<float*>(s_wJ);
#pragma unroll
          for (int b = 0; b < B; ++b) f[b * Q + q] = (float)(wq * J[b]);
        } else {
#pragma unroll
          for (int b = 0; b < B; ++b) s_wJ[b * Q + q] = wq * J[b];
        }
        red[0] = fma(wq, ss, red[0]);
        red[1] = fma(wq, fabs(ss), red[1]);
        red[2] += ok ? 0.0 : 1.0;
      }
      for (int r = lane; r < NM; r += 32) {
        const double t = s_lam[r] * s_uh[r];
        red[3] += t;
        red[4] += fabs(t);
      }
      warp_sums<5>(red);
      __syncwarp();
      const double L0 = red[0] - red[3];
      const double slack = a.slack_rel * (1.0 + red[1] + red[4]);
      // (a3) gradient, lanes over entries
      for (int r = lane; r < NM; r += 32) {
        const int i = r / M, c = r - i * M;
        double acc = 0.0;
        for (int q = 0; q < Q; ++q) acc = fma(Phi[(size_t)q * N + i], s_wu[c * Q + q], acc);
        s_g[r] = acc - s_uh[r];
      }
      __syncwarp();
      double res = 0.0;
      for (int i = lane; i < N; i += 32) {
        double nrm = 0.0;
#pragma unroll
        for (int c = 0; c < M; ++c) nrm = fma(s_g[i * M + c], s_g[i * M + c], nrm);
        res += sqrt(nrm);
      }
      res = warp_sum(res);
      if (red[2] > 0.0) { st = ST_INFEASIBLE; break; }
      if (!isfinite(res)) { st = ST_NONFINITE; break; }
      if (a.one_step) {
        if (it >= 1) break;
      } else {
        if (res < a.tau) break;
        if (it >= a.max_newton) { st = ST_NOCONV; break; }
      }
      // (b) Hessian, lanes over moment pairs (i >= j), all B blocks at once
      for (int pidx = lane; pidx < NP; pidx += 32) {
        const uint32_t pr = a.tab.pairs[pidx];
        const int i = (int)(pr >> 16), j = (int)(pr & 0xffffu);
        double hv[B];
        if (MIXED) {
          const float* f = reinterpret_cast<const float*>(s_wJ);
          float acc[B];
#pragma unroll
          for (int b = 0; b < B; ++b) acc[b] = 0.f;
          for (int q = 0; q < Q; ++q) {
            const float pq = (float)Phi[(size_t)q * N + i] * (float)Phi[(size_t)q * N + j];
#pragma unroll
            for (int b = 0; b < B; ++b) acc[b] = fmaf(f[b * Q + q], pq, acc[b]);
          }
#pragma unroll
          for (int b = 0; b < B; ++b) hv[b] = (double)acc[b];
        } else {
#pragma unroll
          for (int b = 0; b < B; ++b) hv[b] = 0.0;
          for (int q = 0; q < Q; ++q) {
            const double pq = Phi[(size_t)q * N + i] * Phi[(size_t)q * N + j];
#pragma unroll
            for (int b = 0; b < B; ++b) hv[b] = fma(s_wJ[b * Q + q], pq, hv[b]);
          }
        }
#pragma unroll
        for (int a1 = 0; a1 < M; ++a1)
#pragma unroll
          for (int b1 = 0; b1 < M; ++b1) {
            const int r = i * M + a1, c = j * M + b1;
            if (r < c) continue;
            const int lo = a1 < b1 ? a1 : b1, hi = a1 < b1 ? b1 : a1;
            s_H[rowoff_w(r) + c] = hv[packed_ab(lo, hi, M)];
          }
      }
      // gradient as the augmented row NM (the factorisation turns it into L^-1 g)
      for (int r = lane; r < NM; r += 32) s_H[rowoff_w(NM) + r] = s_g[r];
      __syncwarp();
      // (c) right-looking Cholesky, lanes over rows
      bool spd = true;
      for (int k = 0; k < NM; ++k) {
        const double dkk = s_H[rowoff_w(k) + k];
        if (!(dkk > 0.0) || !isfinite(dkk)) { spd = false; break; }
        const double id = rsqrt(dkk);
        __syncwarp();
        if (lane == 0) {
          s_H[rowoff_w(k) + k] = dkk * id;
          s_dinv[k] = id;
        }
        for (int r = k + 1 + lane; r <= NM; r += 32) s_H[rowoff_w(r) + k] *= id;
        __syncwarp();
        // trailing update on an 8 x 4 lane grid (rows x columns), so that the lanes share the
        // triangle evenly (a whole row per lane would leave most lanes idle on the short rows)
        {
          const int ly = lane >> 2, lx = lane & 3;
          for (int r = k + 1 + ly; r <= NM; r += 8) {
            const size_t ro = rowoff_w(r);
            const double lrk = s_H[ro + k];
            const int jmax = r < NM ? r : NM - 1;
            for (int j = k + 1 + lx; j <= jmax; j += 4) s_H[ro + j] = fma(-lrk, s_H[rowoff_w(j) + k], s_H[ro + j]);
          }
        }
        __syncwarp();
      }
      if (!spd) { st = ST_NOTSPD; break; }
      // back substitution L^T Delta = -L^-1 g, one column at a time
      for (int r = lane; r < NM; r += 32) s_d[r] = -s_H[rowoff_w(NM) + r];
      __syncwarp();
      for (int k = NM - 1; k >= 0; --k) {
        const double xk = s_d[k] * s_dinv[k];
        __syncwarp();
        if (lane == 0) s_d[k] = xk;
        const size_t rk = rowoff_w(k);
        for (int r = lane; r < k; r += 32) s_d[r] = fma(-s_H[rk + r], xk, s_d[r]);
        __syncwarp();
      }
      // direction at the nodes, slope, Delta . u_hat
      for (int q = lane; q < Q; q += 32) {
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
      for (int r = lane; r < NM; r += 32) {
        r2[0] = fma(s_g[r], s_d[r], r2[0]);
        r2[1] = fma(s_d[r], s_uh[r], r2[1]);
      }
      warp_sums<2>(r2);
      __syncwarp();
      const double slope = r2[0], dU = r2[1];
      double alpha = 1.0;
      bool accepted = false;
      for (int h = 0; h <= a.max_halvings; ++h) {
        double rr[2] = {0.0, 0.0};
        for (int q = lane; q < Q; q += 32) {
          double L[M], ss;
#pragma unroll
          for (int c = 0; c < M; ++c) L[c] = fma(alpha, s_dLam[c * Q + q], s_Lam[c * Q + q]);
          const bool ok = Closure<ENT, M>::feasible_sstar(L, a.ent, ss);
          rr[0] = fma(w[q], ss, rr[0]);
          rr[1] += ok ? 0.0 : 1.0;
        }
        warp_sums<2>(rr);
        const double Lt = rr[0] - fma(alpha, dU, red[3]);
        if (rr[1] == 0.0 && isfinite(Lt) && Lt <= L0 + a.armijo_c * alpha * slope + slack) {
          accepted = true;
          break;
        }
        alpha *= 0.5;
      }
      if (!accepted) { st = ST_LINESEARCH; break; }
      for (int r = lane; r < NM; r += 32) s_lam[r] = fma(alpha, s_d[r], s_lam[r]);
      __syncwarp();
      ++it;
    }
    for (int r = lane; r < NM; r += 32) lam_g[r] = s_lam[r];
    double* un = a.unode + (size_t)cell * M * Q;
    for (int r = lane; r < M * Q; r += 32) un[r] = s_u[r];
    if (lane == 0) {
      a.iters[cell] = it;
      a.status[cell] = st;
    }
    if (a.track_speed) {
      double smax = 0.0;
      for (int q = lane; q < Q; q += 32) {
        double u[M];
#pragma unroll
        for (int c = 0; c < M; ++c) u[c] = s_u[c * Q + q];
        smax = fmax(smax, node_speed<PHYS, M>(u, a.ent.gamma));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
      if (lane == 0) atomic_max_pos(&a.sc->smax_bits, smax);
    }
    __syncwarp();
    if constexpr (PHYS != PHYS_EULER2D)
      if (a.lf_a) lf_fold_warp<PHYS, M>(a, cell, s_Lam, s_dLam);
  }
}

template <int ENT, int PHYS, int M, bool MIXED>
static cudaError_t launch_w(const NewtonArgs* a, int grid, int warps, int slice, cudaStream_t s, int prepare,
                            int* blocks_per_sm) {
  auto k = k_newton_warp<ENT, PHYS, M, MIXED>;
  const size_t smem = (size_t)warps * slice * sizeof(double);
  if (prepare) {
    cudaError_t e = raise_smem_limit(k, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, 32 * warps, smem);
  }
  k<<<grid, 32 * warps, smem, s>>>(*a, slice);
  return cudaGetLastError();
}

template <typename F>
static cudaError_t dispatch_w(int ent, int phys, int m, bool mixed, F&& f) {
  using std::integral_constant;
  auto go = [&](auto E, auto P, auto MM) {
    return mixed ? f(E, P, MM, std::true_type()) : f(E, P, MM, std::false_type());
  };
  if (phys == PHYS_BURGERS && m == 1) {
    if (ent == ENT_BARRIER) return go(integral_constant<int, ENT_BARRIER>(), integral_constant<int, PHYS_BURGERS>(), integral_constant<int, 1>());
    if (ent == ENT_QUADRATIC) return go(integral_constant<int, ENT_QUADRATIC>(), integral_constant<int, PHYS_BURGERS>(), integral_constant<int, 1>());
  }
  if (phys == PHYS_EULER1D && m == 3) {
    if (ent == ENT_EULER) return go(integral_constant<int, ENT_EULER>(), integral_constant<int, PHYS_EULER1D>(), integral_constant<int, 3>());
    if (ent == ENT_QUADRATIC) return go(integral_constant<int, ENT_QUADRATIC>(), integral_constant<int, PHYS_EULER1D>(), integral_constant<int, 3>());
  }
  if (phys == PHYS_EULER2D && m == 4) {
    if (ent == ENT_EULER) return go(integral_constant<int, ENT_EULER>(), integral_constant<int, PHYS_EULER2D>(), integral_constant<int, 4>());
    if (ent == ENT_QUADRATIC) return go(integral_constant<int, ENT_QUADRATIC>(), integral_constant<int, PHYS_EULER2D>(), integral_constant<int, 4>());
  }
  return cudaErrorInvalidValue;
}

size_t newton_warp_slice(int N, int m, int Q) { return warp_slice_doubles(N, m, Q); }

cudaError_t prepare_newton_warp(int ent, int phys, int m, bool mixed, int warps, int slice, int* blocks_per_sm) {
  return dispatch_w(ent, phys, m, mixed, [&](auto E, auto P, auto MM, auto X) {
    return launch_w<decltype(E)::value, decltype(P)::value, decltype(MM)::value, decltype(X)::value>(
        nullptr, 0, warps, slice, nullptr, 1, blocks_per_sm);
  });
}

cudaError_t launch_newton_warp(int ent, int phys, int m, bool mixed, const NewtonArgs& a, int grid, int warps, int slice,
                               cudaStream_t s) {
  return dispatch_w(ent, phys, m, mixed, [&](auto E, auto P, auto MM, auto X) {
    return launch_w<decltype(E)::value, decltype(P)::value, decltype(MM)::value, decltype(X)::value>(
        &a, grid, warps, slice, s, 0, nullptr);
  });
}

}  // namespace ipm
