// newton_warpq.cu -- the per-cell Newton solve of the IPM dual problem (Sec. 3.1, Eq. L, Eq. tauCrit;
// Sec. 5, Eq. dualIterationFunctionAd on adaptive meshes) for the small cells of an adaptive mesh:
// one warp per cell, the quadrature nodes taken in chunks of 32 (one per lane).
//
// On adaptive meshes most cells sit at the lowest degree (N m <= 64) while the rule has the nodes of
// the finest level (hundreds). The CTA-per-cell kernel spends most of its time in block barriers on
// such cells, and the warp kernel of newton_warp.cu keeps every node's values in shared memory (too
// much per warp at hundreds of nodes). Here a warp streams the nodes in chunks of 32 through a small
// staging area: per chunk the lanes reconstruct Lambda = sum_i lambda_i phi_i(xi_k) at their nodes and
// evaluate the closure; then the lanes, now over gradient entries or moment pairs, add the chunk's
// terms. The Hessian pass recomputes the closure's Jacobian chunk by chunk (a cell that converges
// needs none); the Armijo trials reconstruct Lambda + alpha Delta at the nodes directly. The steps,
// the stopping test and the line search are those of newton.cu; the Cholesky factorisation and the
// back substitution are the lane-grid forms of newton_warp.cu.
//
// Precision. FP64 path: float64 throughout. Mixed path: the Hessian's node sums are FP32 products
// accumulated in FP32 within a chunk, widened and added in float64 across chunks; the gradient,
// stopping test, factorisation, solves and line search stay float64.
//
// Work items: cell_list[*first_dev .. n_work) through the counter *queue (the CTA-per-cell kernel
// takes the items before *first_dev). Every loop is bounded (queue, max_newton, max_halvings, N m).
#include <type_traits>

#include "ipm_host.h"

namespace ipm {

namespace {
constexpr int CHW = 32;   // nodes per chunk (one per lane)

__device__ __forceinline__ size_t rowoff_q(int r) { return (size_t)r * (r + 1) / 2; }

template <int K>
__device__ __forceinline__ void warp_sums_q(double (&v)[K]) {
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = warp_sum(v[k]);
}
}  // namespace

// doubles of one warp's shared-memory slice for cells of up to NM = N m unknowns
__host__ __device__ inline size_t warpq_slice_doubles(int NM, int m) {
  const size_t B = (size_t)m * (m + 1) / 2;
  return 5 * (size_t)NM + (size_t)(m + B) * CHW + (size_t)(NM + 1) * (NM + 2) / 2;
}

template <int ENT, int PHYS, int M, bool MIXED>
__global__ void __launch_bounds__(256) k_newton_warpq(NewtonArgs a, int slice, int nm_slice) {
  constexpr int B = packed_count(M);
  extern __shared__ __align__(16) double qsm[];
  const int NX = a.tab.N, QS = a.tab.Q, NMX = NX * M;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* base = qsm + (size_t)warp * slice;
  double* s_lam = base;
  double* s_uh = s_lam + nm_slice;
  double* s_g = s_uh + nm_slice;
  double* s_d = s_g + nm_slice;
  double* s_dinv = s_d + nm_slice;
  double* s_wu = s_dinv + nm_slice;   // [M][32]  w_k u_k of the chunk
  double* s_wJ = s_wu + M * CHW;      // [B][32]  w_k J_k of the chunk
  double* s_H = s_wJ + B * CHW;       // packed (NM+1)(NM+2)/2
  const double* __restrict__ PhiT = a.tab.PhiT;
  const double* __restrict__ Phi = a.tab.Phi;
  const int first = a.first_dev ? *a.first_dev : 0;
  int* queue = a.queue ? a.queue : &a.sc->work_counter;

  for (;;) {
    int wk = 0;
    if (lane == 0) wk = atomicAdd(queue, 1);
    wk = __shfl_sync(0xffffffffu, wk, 0) + first;
    if (wk >= a.n_work) break;
    const int cell = a.cell_list[wk];
    const int lev = a.level ? a.level[cell] : 0;
    const int N = a.level ? a.lev_n[lev] : NX;
    const int NM = N * M, NP = N * (N + 1) / 2;
    const int Qc = a.lev_w ? a.lev_q[lev] : QS;
    const double* __restrict__ wc = a.lev_w ? a.lev_w + (size_t)lev * QS : a.tab.w;
    double* lam_g = a.lam + (size_t)cell * NMX;
    const double* uh_g = a.uhat + (size_t)cell * NMX;
    double* un = a.unode + (size_t)cell * M * QS;
    for (int r = lane; r < NM; r += 32) {
      s_lam[r] = lam_g[r];
      s_uh[r] = uh_g[r];
    }
    __syncwarp();
    // convergence check from the cell's moment image (as in the CTA-per-cell kernel): S - u_hat with the
    // sums of this kernel's own evaluation, valid while the duals and the level are those it was taken at
    const bool img_rd = a.img != nullptr && !a.one_step && !a.h_dump;
    const bool img_wr = a.img != nullptr && !a.h_dump;
    if (img_rd) {
      bool same = a.img_valid[cell] == lev + 1;
      if (same) {
        const double* Sc = a.img + (size_t)cell * NMX;
        const double* Lc = a.img_lam + (size_t)cell * NMX;
        for (int r = lane; r < NM; r += 32) {
          same = same && __double_as_longlong(Lc[r]) == __double_as_longlong(s_lam[r]);
          s_g[r] = Sc[r] - s_uh[r];
        }
      }
      if (__all_sync(0xffffffffu, same)) {
        __syncwarp();
        double res = 0.0;
        for (int i = lane; i < N; i += 32) {
          double nrm = 0.0;
#pragma unroll
          for (int c = 0; c < M; ++c) nrm = fma(s_g[i * M + c], s_g[i * M + c], nrm);
          res += sqrt(nrm);
        }
        res = warp_sum(res);
        if (res < a.tau) {
          if (lane == 0) {
            a.iters[cell] = 0;
            a.status[cell] = ST_OK;
            atomicAdd(&a.sc->cached_checks, 1ULL);
            if (a.track_speed) atomic_max_pos(&a.sc->smax_bits, a.img_smax[cell]);
          }
          __syncwarp();
          continue;
        }
      }
    }
    if (a.img != nullptr && lane == 0) a.img_valid[cell] = 0;
    __syncwarp();
    int it = 0, st = ST_OK;
    for (;;) {
      // (a1)-(a3): reconstruction and closure per node, cost terms, gradient sums chunk by chunk; the
      // nodal states of every evaluation are written out (the last one belongs to the final duals)
      double red[5] = {0.0, 0.0, 0.0, 0.0, 0.0};  // sum w s*, sum w |s*|, #infeasible, lambda.uhat, sum |lambda uhat|
      for (int r = lane; r < NM; r += 32) s_g[r] = 0.0;
      for (int q0 = 0; q0 < Qc; q0 += CHW) {
        const int q = q0 + lane;
        double wu[M];
        if (q < Qc) {
          double L[M], u[M], ss;
#pragma unroll
          for (int c = 0; c < M; ++c) L[c] = 0.0;
          for (int i = 0; i < N; ++i) {
            const double ph = PhiT[(size_t)i * QS + q];
#pragma unroll
            for (int c = 0; c < M; ++c) L[c] = fma(ph, s_lam[i * M + c], L[c]);
          }
          const bool ok = Closure<ENT, M>::template eval<false>(L, a.ent, u, nullptr, ss);
          const double wq = wc[q];
#pragma unroll
          for (int c = 0; c < M; ++c) {
            wu[c] = wq * u[c];
            un[c * QS + q] = u[c];
          }
          red[0] = fma(wq, ss, red[0]);
          red[1] = fma(wq, fabs(ss), red[1]);
          red[2] += ok ? 0.0 : 1.0;
        } else {
#pragma unroll
          for (int c = 0; c < M; ++c) wu[c] = 0.0;
        }
#pragma unroll
        for (int c = 0; c < M; ++c) s_wu[c * CHW + lane] = wu[c];
        __syncwarp();
        const int nq = min(CHW, Qc - q0);
        for (int r = lane; r < NM; r += 32) {
          const int i = r / M, c = r - i * M;
          double acc = s_g[r];
          for (int l = 0; l < nq; ++l) acc = fma(Phi[(size_t)(q0 + l) * NX + i], s_wu[c * CHW + l], acc);
          s_g[r] = acc;
        }
        __syncwarp();
      }
      for (int r = lane; r < NM; r += 32) {
        const double t = s_lam[r] * s_uh[r];
        red[3] += t;
        red[4] += fabs(t);
        if (img_wr) a.img[(size_t)cell * NMX + r] = s_g[r];
        s_g[r] -= s_uh[r];
      }
      warp_sums_q<5>(red);
      __syncwarp();
      const double L0 = red[0] - red[3];
      const double slack = a.slack_rel * (1.0 + red[1] + red[4]);
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
      // (b) Hessian: closure Jacobians chunk by chunk, lanes over moment pairs (i >= j), all B blocks
      const size_t nh = rowoff_q(NM);
      for (size_t r = lane; r < nh; r += 32) s_H[r] = 0.0;
      __syncwarp();
      for (int q0 = 0; q0 < Qc; q0 += CHW) {
        const int q = q0 + lane;
        double wJ[B];
        if (q < Qc) {
          double L[M], u[M], J[B], ss;
#pragma unroll
          for (int c = 0; c < M; ++c) L[c] = 0.0;
          for (int i = 0; i < N; ++i) {
            const double ph = PhiT[(size_t)i * QS + q];
#pragma unroll
            for (int c = 0; c < M; ++c) L[c] = fma(ph, s_lam[i * M + c], L[c]);
          }
          Closure<ENT, M>::template eval<true>(L, a.ent, u, J, ss);
          const double wq = wc[q];
#pragma unroll
          for (int b = 0; b < B; ++b) wJ[b] = wq * J[b];
        } else {
#pragma unroll
          for (int b = 0; b < B; ++b) wJ[b] = 0.0;
        }
#pragma unroll
        for (int b = 0; b < B; ++b) s_wJ[b * CHW + lane] = wJ[b];
        __syncwarp();
        const int nq = min(CHW, Qc - q0);
        for (int pidx = lane; pidx < NP; pidx += 32) {
          const uint32_t pr = a.tab.pairs[pidx];
          const int i = (int)(pr >> 16), j = (int)(pr & 0xffffu);
          double hv[B];
          if (MIXED) {
            float acc[B];
#pragma unroll
            for (int b = 0; b < B; ++b) acc[b] = 0.f;
            for (int l = 0; l < nq; ++l) {
              const size_t ro = (size_t)(q0 + l) * NX;
              const float pq = (float)Phi[ro + i] * (float)Phi[ro + j];
#pragma unroll
              for (int b = 0; b < B; ++b) acc[b] = fmaf((float)s_wJ[b * CHW + l], pq, acc[b]);
            }
#pragma unroll
            for (int b = 0; b < B; ++b) hv[b] = (double)acc[b];
          } else {
#pragma unroll
            for (int b = 0; b < B; ++b) hv[b] = 0.0;
            for (int l = 0; l < nq; ++l) {
              const size_t ro = (size_t)(q0 + l) * NX;
              const double pq = Phi[ro + i] * Phi[ro + j];
#pragma unroll
              for (int b = 0; b < B; ++b) hv[b] = fma(s_wJ[b * CHW + l], pq, hv[b]);
            }
          }
#pragma unroll
          for (int a1 = 0; a1 < M; ++a1)
#pragma unroll
            for (int b1 = 0; b1 < M; ++b1) {
              const int r = i * M + a1, c = j * M + b1;
              if (r < c) continue;
              const int lo = a1 < b1 ? a1 : b1, hi = a1 < b1 ? b1 : a1;
              s_H[rowoff_q(r) + c] += hv[packed_ab(lo, hi, M)];
            }
        }
        __syncwarp();
      }
      // gradient as the augmented row NM (the factorisation turns it into L^-1 g)
      for (int r = lane; r < NM; r += 32) s_H[rowoff_q(NM) + r] = s_g[r];
      __syncwarp();
      // (c) right-looking Cholesky, trailing updates on an 8 x 4 lane grid (rows x columns)
      bool spd = true;
      for (int k = 0; k < NM; ++k) {
        const double dkk = s_H[rowoff_q(k) + k];
        if (!(dkk > 0.0) || !isfinite(dkk)) { spd = false; break; }
        const double id = rsqrt(dkk);
        __syncwarp();
        if (lane == 0) {
          s_H[rowoff_q(k) + k] = dkk * id;
          s_dinv[k] = id;
        }
        for (int r = k + 1 + lane; r <= NM; r += 32) s_H[rowoff_q(r) + k] *= id;
        __syncwarp();
        {
          const int ly = lane >> 2, lx = lane & 3;
          for (int r = k + 1 + ly; r <= NM; r += 8) {
            const size_t ro = rowoff_q(r);
            const double lrk = s_H[ro + k];
            const int jmax = r < NM ? r : NM - 1;
            for (int j = k + 1 + lx; j <= jmax; j += 4) s_H[ro + j] = fma(-lrk, s_H[rowoff_q(j) + k], s_H[ro + j]);
          }
        }
        __syncwarp();
      }
      if (!spd) { st = ST_NOTSPD; break; }
      // back substitution L^T Delta = -L^-1 g, one column at a time
      for (int r = lane; r < NM; r += 32) s_d[r] = -s_H[rowoff_q(NM) + r];
      __syncwarp();
      for (int k = NM - 1; k >= 0; --k) {
        const double xk = s_d[k] * s_dinv[k];
        __syncwarp();
        if (lane == 0) s_d[k] = xk;
        const size_t rk = rowoff_q(k);
        for (int r = lane; r < k; r += 32) s_d[r] = fma(-s_H[rk + r], xk, s_d[r]);
        __syncwarp();
      }
      double r2[2] = {0.0, 0.0};
      for (int r = lane; r < NM; r += 32) {
        r2[0] = fma(s_g[r], s_d[r], r2[0]);
        r2[1] = fma(s_d[r], s_uh[r], r2[1]);
      }
      warp_sums_q<2>(r2);
      __syncwarp();
      const double slope = r2[0], dU = r2[1];
      // Armijo backtracking; the trial Lambda + alpha Delta is reconstructed at each node
      double alpha = 1.0;
      bool accepted = false;
      for (int h = 0; h <= a.max_halvings; ++h) {
        double rr[2] = {0.0, 0.0};
        for (int q = lane; q < Qc; q += 32) {
          double L[M], D[M], ss;
#pragma unroll
          for (int c = 0; c < M; ++c) L[c] = D[c] = 0.0;
          for (int i = 0; i < N; ++i) {
            const double ph = PhiT[(size_t)i * QS + q];
#pragma unroll
            for (int c = 0; c < M; ++c) {
              L[c] = fma(ph, s_lam[i * M + c], L[c]);
              D[c] = fma(ph, s_d[i * M + c], D[c]);
            }
          }
#pragma unroll
          for (int c = 0; c < M; ++c) L[c] = fma(alpha, D[c], L[c]);
          const bool ok = Closure<ENT, M>::feasible_sstar(L, a.ent, ss);
          rr[0] = fma(wc[q], ss, rr[0]);
          rr[1] += ok ? 0.0 : 1.0;
        }
        warp_sums_q<2>(rr);
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
    // nodal states beyond this cell's rule that the stencil's updates read (per-level rules), zero
    // beyond them; then the wave speed at the nodes of the rule of the cell's new level
    const int qe = a.q_eval ? a.q_eval[cell] : Qc;
    for (int q = min(Qc, qe) + lane; q < QS; q += 32) {
      double u[M];
      if (q < qe) {
        double L[M], ss;
#pragma unroll
        for (int c = 0; c < M; ++c) L[c] = 0.0;
        for (int i = 0; i < N; ++i) {
          const double ph = PhiT[(size_t)i * QS + q];
#pragma unroll
          for (int c = 0; c < M; ++c) L[c] = fma(ph, s_lam[i * M + c], L[c]);
        }
        Closure<ENT, M>::template eval<false>(L, a.ent, u, nullptr, ss);
      } else {
#pragma unroll
        for (int c = 0; c < M; ++c) u[c] = 0.0;
      }
#pragma unroll
      for (int c = 0; c < M; ++c) un[c * QS + q] = u[c];
    }
    __syncwarp();
    if (lane == 0) {
      a.iters[cell] = it;
      a.status[cell] = st;
    }
    const bool keep_img = img_wr && st == ST_OK;
    if (keep_img)
      for (int r = lane; r < NM; r += 32) a.img_lam[(size_t)cell * NMX + r] = s_lam[r];
    if (a.track_speed || keep_img) {
      const int qs = (a.lev_w && a.level_next) ? a.lev_q[a.level_next[cell]] : Qc;
      double smax = 0.0;
      for (int q = lane; q < qs; q += 32) {
        double u[M];
#pragma unroll
        for (int c = 0; c < M; ++c) u[c] = un[c * QS + q];
        smax = fmax(smax, node_speed<PHYS, M>(u, a.ent.gamma));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
      if (lane == 0) {
        if (a.track_speed) atomic_max_pos(&a.sc->smax_bits, smax);
        if (keep_img) {
          a.img_smax[cell] = smax;
          a.img_valid[cell] = lev + 1;
        }
      }
    }
    __syncwarp();
  }
}

template <int ENT, int PHYS, int M, bool MIXED>
static cudaError_t launch_wq(const NewtonArgs* a, int grid, int warps, int slice, int nm_slice, cudaStream_t s,
                             int prepare, int* blocks_per_sm) {
  auto k = k_newton_warpq<ENT, PHYS, M, MIXED>;
  const size_t smem = (size_t)warps * slice * sizeof(double);
  if (prepare) {
    cudaError_t e = raise_smem_limit(k, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, 32 * warps, smem);
  }
  k<<<grid, 32 * warps, smem, s>>>(*a, slice, nm_slice);
  return cudaGetLastError();
}

template <typename F>
static cudaError_t dispatch_wq(int ent, int phys, int m, bool mixed, F&& f) {
  using std::integral_constant;
  auto go = [&](auto E, auto P, auto MM) {
    return mixed ? f(E, P, MM, std::true_type()) : f(E, P, MM, std::false_type());
  };
  // adaptive meshes are 2-D Euler
  if (phys == PHYS_EULER2D && m == 4) {
    if (ent == ENT_EULER) return go(integral_constant<int, ENT_EULER>(), integral_constant<int, PHYS_EULER2D>(), integral_constant<int, 4>());
    if (ent == ENT_QUADRATIC) return go(integral_constant<int, ENT_QUADRATIC>(), integral_constant<int, PHYS_EULER2D>(), integral_constant<int, 4>());
  }
  return cudaErrorInvalidValue;
}

size_t newton_warpq_slice(int nm, int m) { return warpq_slice_doubles(nm, m); }

cudaError_t prepare_newton_warpq(int ent, int phys, int m, bool mixed, int warps, int slice, int* blocks_per_sm) {
  return dispatch_wq(ent, phys, m, mixed, [&](auto E, auto P, auto MM, auto X) {
    return launch_wq<decltype(E)::value, decltype(P)::value, decltype(MM)::value, decltype(X)::value>(
        nullptr, 0, warps, slice, 0, nullptr, 1, blocks_per_sm);
  });
}

cudaError_t launch_newton_warpq(int ent, int phys, int m, bool mixed, const NewtonArgs& a, int grid, int warps,
                                int slice, int nm_slice, cudaStream_t s) {
  return dispatch_wq(ent, phys, m, mixed, [&](auto E, auto P, auto MM, auto X) {
    return launch_wq<decltype(E)::value, decltype(P)::value, decltype(MM)::value, decltype(X)::value>(
        &a, grid, warps, slice, nm_slice, s, 0, nullptr);
  });
}

}  // namespace ipm
