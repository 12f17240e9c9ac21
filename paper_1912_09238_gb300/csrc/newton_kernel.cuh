// newton_kernel.cuh -- the per-cell Newton solve of the IPM dual problem as one kernel template
// (k_newton) and its launch helpers; each precision / factorisation mode is instantiated in its own
// translation unit (newton_m0.cu .. newton_m4.cu) so that the variants compile in parallel.
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
// Precision. FP64 path: every step in float64 on the CUDA cores. Mixed path: only (b) changes.
// For each packed pair ab (a <= b) the block H_ab = Phi^T diag(w J_ab) Phi is one tensor-core
// contraction over the nodes: the per-cell operand A[(ab, i)][k] = w_k J_k,ab phi_i(xi_k) and the
// constant operand B[j][k] = phi_j(xi_k) are each split into two BF16 terms (x = x_hi + x_lo,
// |x - x_hi - x_lo| <= 2^-16 |x|), and A_hi B_hi + A_hi B_lo + A_lo B_hi is accumulated in FP32 in
// tensor memory by tcgen05.mma. The result is widened to float64 for the Cholesky factorisation.
// The gradient, the stopping test, the factorisation, the solves and the line search stay in
// float64, so the converged duals satisfy the same FP64 criterion (Eq. tauCrit) as the FP64 path.
//
// Every loop is bounded: the queue by the cell count, Newton by max_newton, the line search by
// max_halvings, the factorisation and solves by N*m, and every tensor-core / bulk-copy wait by a
// 2 s global-timer limit (a timeout marks the cell IPM_ETIMEOUT, counts in StepScalars::tc_timeouts
// and ends the CTA after draining its pending copies).
#pragma once
#include <type_traits>

#include <cuda_bf16.h>

#include "ipm_host.h"
#include "tc.cuh"

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

// Stopping quantity of Eq. tauCrit: sum over the moments i of the 2-norm of g_i over the variables
// (block-wide; every thread returns it)
template <int M>
__device__ __forceinline__ double grad_residual(const double* s_g, int N, double* s_red) {
  double gres[1] = {0.0};
  for (int i = threadIdx.x; i < N; i += NT) {
    double nrm = 0.0;
#pragma unroll
    for (int c = 0; c < M; ++c) nrm = fma(s_g[i * M + c], s_g[i * M + c], nrm);
    gres[0] += sqrt(nrm);
  }
  block_sum<1>(gres, s_red);
  return gres[0];
}

// (a, b) of the packed index ab (a <= b)
template <int M>
__device__ __forceinline__ void unpack_ab(int ab, int& a, int& b) {
  a = 0;
  b = 0;
#pragma unroll
  for (int x = 0; x < M; ++x)
#pragma unroll
    for (int y = x; y < M; ++y)
      if (packed_ab(x, y, M) == ab) {
        a = x;
        b = y;
      }
}

// Store the value H_ab[i][j] (a <= b) of the block form into the packed lower triangle of H
// (row index i*M + a). Each lower entry is written by exactly one (ab, i, j).
template <int M, typename T>
__device__ __forceinline__ void store_block_entry(T* s_H, int a, int b, int i, int j, T v) {
  if (a == b) {
    if (i >= j) {
      const size_t r = (size_t)i * M + a, c = (size_t)j * M + a;
      s_H[r * (r + 1) / 2 + c] = v;
    }
  } else {
    if (i > j) {
      const size_t r = (size_t)i * M + a, c = (size_t)j * M + b;
      s_H[r * (r + 1) / 2 + c] = v;
    }
    if (i >= j) {
      const size_t r = (size_t)i * M + b, c = (size_t)j * M + a;
      s_H[r * (r + 1) / 2 + c] = v;
    }
  }
}

// (b), FP64 on the CUDA cores: one thread per moment pair (i >= j), all B blocks at once.
template <int M>
__device__ __forceinline__ void hessian_fp64(const NewtonArgs& a, int N, int Qc, const double* s_wJ, double* s_H) {
  constexpr int B = packed_count(M);
  const int ldN = a.tab.N, Q = a.tab.Q, NP = N * (N + 1) / 2;
  const double* __restrict__ Phi = a.tab.Phi;
  for (int pidx = threadIdx.x; pidx < NP; pidx += NT) {
    const uint32_t pr = a.tab.pairs[pidx];
    const int i = (int)(pr >> 16), j = (int)(pr & 0xffffu);
    double acc[B];
#pragma unroll
    for (int b = 0; b < B; ++b) acc[b] = 0.0;
    for (int q = 0; q < Qc; ++q) {
      const double pq = Phi[(size_t)q * ldN + i] * Phi[(size_t)q * ldN + j];
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
}

// ------------------------------------------------------------------------------------------------
// (c) Blocked Cholesky factorisation with the forward substitution folded in.
//
// A is the packed lower triangle (row r at offset r(r+1)/2) of the (n+1) x (n+1) matrix
// [[H, .], [g^T, .]]: rows 0..n-1 hold H, row n holds the gradient g. Factorising the leading n x n
// block H = L L^T right-looking also turns row n into y = L^-1 g (the forward substitution), because
// row n takes part in every scaling and trailing update but is never a pivot.
// Panels of NB columns: (1) the NB x NB diagonal block is factorised by one warp with its rows in
// registers; (2) every row below it (row n included) is solved against that block by one thread;
// (3) the trailing rows and columns are updated with a rank-NB product, 2 x 2 outputs per thread.
// s_P holds the current panel's columns row by row (stride PSTR), s_dinv the reciprocal pivots.
// Returns false if a pivot is not positive and finite (H not numerically SPD).
// ------------------------------------------------------------------------------------------------
constexpr int NB = 8;
constexpr int PSTR = NB + 1;

__device__ __forceinline__ size_t rowoff(int r) { return (size_t)r * (r + 1) / 2; }
// cell index of work item w on the interior of an (nx+2)-wide mesh with one ghost layer, starting at row gy
__device__ __forceinline__ int work_cell(int w, int nx, int gy) { return (w / nx + gy) * (nx + 2) + (w % nx + 1); }

// element-type helpers of the factorisation (T = double, or float for the FP32-factor mode)
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }

// A[r][c] -= sum_k P[r][k] P[c][k] for rows r0..r0+3 (<= n) and columns c0, c0+1 (< n, <= r).
// KW = NB: full panel (no guards on k); KW = 0: kw columns.
template <int KW, typename T>
__device__ __forceinline__ void trailing_tile(T* A, const T* s_P, int n, int r0, int c0, int kw) {
  T acc[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = (T)0;
  bool rv[4], cv[2];
#pragma unroll
  for (int i = 0; i < 4; ++i) rv[i] = r0 + i <= n;
#pragma unroll
  for (int j = 0; j < 2; ++j) cv[j] = c0 + j < n;
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    if (KW == NB || k < kw) {
      T p[4], q[2];
#pragma unroll
      for (int i = 0; i < 4; ++i) p[i] = rv[i] ? s_P[(r0 + i) * PSTR + k] : (T)0;
#pragma unroll
      for (int j = 0; j < 2; ++j) q[j] = cv[j] ? s_P[(c0 + j) * PSTR + k] : (T)0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) acc[i][j] = fma(p[i], q[j], acc[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j)
      if (rv[i] && cv[j] && c0 + j <= r0 + i) A[rowoff(r0 + i) + c0 + j] -= acc[i][j];
}

// Factorise the NB x NB diagonal block at rows/columns kb..kb+kw-1 (already updated by all earlier
// panels); called by one full warp, lane i owning row kb + i in registers. Writes L into A and into
// the panel buffer P, the reciprocal pivots into s_dinv; sets *s_flag on a bad pivot.
template <typename T>
__device__ __forceinline__ void panel_diag(T* A, int kb, int kw, T* P, T* s_dinv, int* s_flag) {
  const int lane = threadIdx.x & 31;
  T row[NB];
  const bool mine = lane < kw;
#pragma unroll
  for (int j = 0; j < NB; ++j) row[j] = (mine && j <= lane) ? A[rowoff(kb + lane) + kb + j] : (T)0;
  bool ok = true;
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    if (k < kw) {
      const T dkk = __shfl_sync(0xffffffffu, row[k], k);
      ok = ok && dkk > (T)0 && isfinite(dkk);
      const T id = rsqrt_t(dkk > (T)0 ? dkk : (T)1);
      if (lane == k) row[k] = dkk * id;
      if (lane > k) row[k] *= id;
#pragma unroll
      for (int j = k + 1; j < NB; ++j) {
        if (j < kw) {
          const T ljk = __shfl_sync(0xffffffffu, row[k], j);
          if (lane >= j) row[j] = fma(-row[k], ljk, row[j]);
        }
      }
      if (lane == 0) s_dinv[kb + k] = id;
    }
  }
  if (mine) {
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      if (j <= lane) {
        A[rowoff(kb + lane) + kb + j] = row[j];
        P[(kb + lane) * PSTR + j] = row[j];
      }
    }
  }
  if (lane == 0 && !ok) *s_flag = 1;
}

// Rows r = kb+kw .. n of the panel: L[r][kb..kb+kw) = A[r][kb..kb+kw) L_bb^-T, by threads t0, t0+stride, ...
template <typename T>
__device__ __forceinline__ void panel_trsm(T* A, int n, int kb, int kw, T* P, const T* s_dinv, int t0,
                                           int stride) {
  for (int r = kb + kw + t0; r <= n; r += stride) {
    const size_t ro = rowoff(r) + kb;
    T x[NB];
#pragma unroll
    for (int k = 0; k < NB; ++k) {
      if (k < kw) {
        T v = A[ro + k];
#pragma unroll
        for (int j = 0; j < k; ++j) v = fma(-x[j], P[(kb + k) * PSTR + j], v);
        x[k] = v * s_dinv[kb + k];
      }
    }
#pragma unroll
    for (int k = 0; k < NB; ++k) {
      if (k < kw) {
        A[ro + k] = x[k];
        P[r * PSTR + k] = x[k];
      }
    }
  }
}

// Rank-kw update with panel P of rows s1..n and columns s1..min(r, n-1), tiles of 4 rows x 2 columns,
// by threads t0, t0+stride, ...
template <typename T>
__device__ __forceinline__ void trailing_update(T* A, int n, const T* P, int kw, int s1, int t0, int stride) {
  const int TR = (n + 4 - s1) / 4;                // row tiles (rows s1..n)
  const int ntiles = TR * (TR + 1);               // row tile ti has 2 ti + 2 column tiles
  for (int t = t0; t < ntiles; t += stride) {
    int ti = (int)((sqrtf(4.f * (float)t + 1.f) - 1.f) * 0.5f);
    while (ti > 0 && ti * (ti + 1) > t) --ti;
    while ((ti + 1) * (ti + 2) <= t) ++ti;
    const int r0 = s1 + 4 * ti, c0 = s1 + 2 * (t - ti * (ti + 1));
    if (c0 >= n) continue;
    if (kw == NB) trailing_tile<NB>(A, P, n, r0, c0, kw);
    else trailing_tile<0>(A, P, n, r0, c0, kw);
  }
}

// Blocked right-looking Cholesky with one panel of look-ahead. s_P holds two panel buffers of
// (n+1) x PSTR. Per panel p: (A) all threads apply panel p to the columns of panel p+1; then
// (B) warp 0 factorises panel p+1 (diagonal block, then its rows below) while warps 1.. apply
// panel p to the rest of the trailing matrix. The latency-bound diagonal block thus overlaps the
// FP64-throughput-bound trailing update.
template <typename T>
__device__ bool cholesky_aug(T* A, int n, T* s_P, T* s_dinv, int* s_flag) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int pbuf = (n + 1) * PSTR;
  if (tid == 0) *s_flag = 0;
  __syncthreads();
  {
    const int kw0 = min(NB, n);
    if (warp == 0) panel_diag(A, 0, kw0, s_P, s_dinv, s_flag);
    __syncthreads();
    if (*s_flag) return false;
    panel_trsm(A, n, 0, kw0, s_P, s_dinv, tid, NT);
    __syncthreads();
  }
  int p = 0;
  for (int kb = 0; kb < n; kb += NB, ++p) {
    const int kw = min(NB, n - kb), s0 = kb + kw;
    if (s0 >= n) break;                            // only the gradient row is left: nothing to update
    const T* P = s_P + (p & 1) * pbuf;
    T* Pn = s_P + ((p + 1) & 1) * pbuf;
    const int kw1 = min(NB, n - s0);
    // (A) columns s0 .. s0+kw1-1 of rows s0..n
    const int rows = n + 1 - s0;
    for (int item = tid; item < rows * kw1; item += NT) {
      const int r = s0 + item / kw1, c = s0 + item % kw1;
      if (c > r) continue;
      T acc = (T)0;
#pragma unroll
      for (int k = 0; k < NB; ++k)
        if (k < kw) acc = fma(P[r * PSTR + k], P[c * PSTR + k], acc);
      A[rowoff(r) + c] -= acc;
    }
    __syncthreads();
    // (B)
    if (warp == 0) {
      panel_diag(A, s0, kw1, Pn, s_dinv, s_flag);
      __syncwarp();
      panel_trsm(A, n, s0, kw1, Pn, s_dinv, lane, 32);
    } else {
      trailing_update(A, n, P, kw, s0 + kw1, tid - 32, NT - 32);
    }
    __syncthreads();
    if (*s_flag) return false;
  }
  return true;
}

// Forward substitution L y = b in place on x (x holds b on entry), blocks of NB from the top: one
// warp solves the diagonal block (lane i holds entry kb + i), then all threads update the rows below.
// Used when a stored factor is reused (the factorisation itself folds the forward solve in).
template <typename T>
__device__ void forward_substitute(const T* A, int n, const T* s_dinv, T* x) {
  const int tid = threadIdx.x, lane = tid & 31;
  for (int kb = 0; kb < n; kb += NB) {
    const int kw = min(NB, n - kb);
    if (tid < 32) {
      T v = lane < kw ? x[kb + lane] : (T)0;
#pragma unroll
      for (int k = 0; k < NB; ++k) {
        if (k < kw) {
          const T yk = __shfl_sync(0xffffffffu, v, k) * s_dinv[kb + k];
          if (lane == k) v = yk;
          if (lane > k && lane < kw) v = fma(-A[rowoff(kb + lane) + kb + k], yk, v);
        }
      }
      if (lane < kw) x[kb + lane] = v;
    }
    __syncthreads();
    for (int r = kb + kw + tid; r < n; r += NT) {
      const size_t ro = rowoff(r) + kb;
      T v = x[r];
#pragma unroll
      for (int k = 0; k < NB; ++k)
        if (k < kw) v = fma(-A[ro + k], x[kb + k], v);
      x[r] = v;
    }
    __syncthreads();
  }
}

// Diagonal block of the back substitution, one warp: lane i holds entry kb + i of the right-hand side
// in v on entry and of the solution on exit (lanes >= kw: unused).
template <typename T>
__device__ __forceinline__ T back_diag(const T* A, int kb, int kw, const T* s_dinv, T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = NB - 1; k >= 0; --k) {
    if (k < kw) {
      const T xk = __shfl_sync(0xffffffffu, v, k) * s_dinv[kb + k];
      if (lane == k) v = xk;
      if (lane < k) v = fma(-A[rowoff(kb + k) + kb + lane], xk, v);
    }
  }
  return v;
}

// Back substitution L^T x = b in place on x (x holds b on entry), blocks of NB from the bottom, with
// one block of look-ahead: once block kb is solved, warp 0 applies it to the NB entries of the next
// block up and solves that block's diagonal, while warps 1.. apply it to all entries above those.
// Every entry receives the same products in the same order as without the look-ahead.
template <typename T>
__device__ void back_substitute(const T* A, int n, const T* s_dinv, T* x) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int kb = ((n - 1) / NB) * NB;
  if (warp == 0) {
    const int kw = min(NB, n - kb);
    const T v = back_diag(A, kb, kw, s_dinv, lane < kw ? x[kb + lane] : (T)0);
    if (lane < kw) x[kb + lane] = v;
  }
  __syncthreads();
  while (kb > 0) {
    const int kw = min(NB, n - kb), kb1 = kb - NB;   // the blocks above the last one are full
    if (warp == 0) {
      T v = (T)0;
      if (lane < NB) {
        v = x[kb1 + lane];
#pragma unroll
        for (int k = 0; k < NB; ++k)
          if (k < kw) v = fma(-A[rowoff(kb + k) + kb1 + lane], x[kb + k], v);
      }
      v = back_diag(A, kb1, NB, s_dinv, v);
      if (lane < NB) x[kb1 + lane] = v;
    } else {
      for (int r = tid - 32; r < kb1; r += NT - 32) {
        T v = x[r];
#pragma unroll
        for (int k = 0; k < NB; ++k)
          if (k < kw) v = fma(-A[rowoff(kb + k) + r], x[kb + k], v);
        x[r] = v;
      }
    }
    __syncthreads();
    kb = kb1;
  }
}

// Tensor-core pipeline state of one CTA (uniform across its threads).
struct TcState {
  uint64_t* bars;     // [0] Hessian MMA completion, [1], [2] Phi chunk buffers, [3], [4] split-factor MMA sets,
                      // [5], [6] staged Phi^T chunk buffers
  uint32_t tmem;      // tensor-memory base address
  uint32_t ph[7];     // parity of the next phase to wait for, per barrier
  bool pend[7];       // a phase is outstanding on the barrier
};
constexpr int TC_BARS = 7;

__device__ __forceinline__ bool tc_wait(TcState& t, int k) {
  const bool ok = tc::mbar_wait(&t.bars[k], t.ph[k]);
  if (ok) {
    t.ph[k] ^= 1u;
    t.pend[k] = false;
  }
  return ok;
}

// FP32 -> T. For T = double the conversion is exact and done on the integer pipes from the IEEE formats
// (a subnormal FP32 value, below 1.2e-38 in magnitude, becomes zero): the FP64 pipe is the scarce one.
template <typename T>
__device__ __forceinline__ T widen(float f);
template <>
__device__ __forceinline__ float widen<float>(float f) { return f; }
template <>
__device__ __forceinline__ double widen<double>(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xFFu;
  const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
  if (e == 0) return __longlong_as_double((long long)sign);
  const unsigned long long ex = e == 0xFFu ? 0x7FFull : (unsigned long long)(e + 896u);   // e - 127 + 1023
  return __longlong_as_double((long long)(sign | (ex << 52) | ((unsigned long long)(b & 0x7FFFFFu) << 29)));
}

// (b), mixed: split-BF16 products on the tensor cores, FP32 accumulate in tensor memory, then
// widened into the packed FP64 H. s_wJf holds w_k J_k,ab as float [B][Q]. Returns false when a
// bounded wait ran out (the CTA must stop).
// s_ph: room for two staged chunks of Phi^T (FP32, n_rows x kcp each) or nullptr. When given, every
// K-chunk's Phi^T columns arrive by bulk copy one chunk ahead of the build that reads them; otherwise
// the build reads Phi^T from global memory (L2). UNROLL: items per thread in flight in the build (2 on
// the one-CTA-per-SM split kernels, 1 where the register budget is halved for two CTAs per SM).
// Warp 0 issues the MMAs (lane 0) and the bulk copies; warps 1..7 build the A operand, so the MMA issue
// of chunk c overlaps the build of chunk c + 1. With mx.stack (chosen once per layout) and the cell's N
// the table's, B = [B_hi; B_lo] is one operand of 2 n_pad rows: A_hi B_hi and A_hi B_lo come from one MMA
// into adjacent accumulators and A_lo B_hi is added to the first, two MMAs per K-step instead of three;
// the two accumulators are added in the epilogue.
template <int M, typename T, int UNROLL>
__device__ bool hessian_tc(const NewtonArgs& a, int N, int Qc, const float* s_wJf, T* s_H, uint8_t* sA, uint8_t* sB,
                           float* s_ph, TcState& t, int* s_abort) {
  constexpr int B = packed_count(M);
  const MixedTiles& mx = a.mx;
  const int Q = a.tab.Q, BN = B * N;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t sbo = tc::kmajor_sbo(mx.kc);
  const uint32_t a_img = (uint32_t)mx.tpp * 128u * (uint32_t)mx.kc * 2u;   // one BF16 term of A
  const uint32_t b_img = (uint32_t)mx.n_pad * (uint32_t)mx.kc * 2u;         // one BF16 term of B (table size)
  const uint32_t b_chunk = 2u * b_img;
  const uint32_t a_buf = 2u * a_img;                                         // both terms of one chunk
  const bool two_a = mx.abuf == 2;
  // this cell's tiling (N may be below the table's on adaptive meshes: the Phi image rows beyond N
  // only feed accumulator columns that are never read back)
  const int n_pad = (N + 15) / 16 * 16;
  const int tiles = (BN + 127) / 128;
  const int tpp = min(mx.tpp, tiles);
  const bool stack = mx.stack && n_pad == mx.n_pad;                       // the cell's N is the table's
  const int acc_cols = stack ? 2 * n_pad : n_pad;                            // tensor-memory columns per row tile
  const uint32_t idesc = tc::idesc_bf16_f32(128, n_pad);
  const uint32_t idesc2 = tc::idesc_bf16_f32(128, 2 * n_pad);
  const int groups = mx.kc / 8;
  // K chunks of this cell's rule (a prefix of the table's nodes; the rest of the last chunk is zero in A)
  const int chunks = (Qc + mx.kc - 1) / mx.kc;
  const bool staged = s_ph != nullptr;
  const int kcp = mx.kcp;
  // item -> (row, group of 8 nodes) by shifts (kc is 16 or 32), row -> (ab, i) by a multiply-high:
  // floor(R / N) = umulhi(R, ceil(2^32 / N)) exactly for R N < 2^32
  const int gshift = groups == 4 ? 2 : 1;
  const uint32_t inv_n = 0xFFFFFFFFu / (uint32_t)N + 1u;
  // w J rows read as float4 when they are 16-byte aligned (the last group of a row may read up to seven
  // floats past Qc: entries of the next row or of the shared-memory region after it, all masked below)
  const bool wj_vec = (Q & 3) == 0 && (reinterpret_cast<uintptr_t>(s_wJf) & 15u) == 0;
  const uint32_t ph_floats = (uint32_t)mx.n_rows * (uint32_t)kcp;
  const uint32_t ph_bytes = ph_floats * 4u;

  for (int t0 = 0; t0 < tiles; t0 += tpp) {
    const int nt = min(tpp, tiles - t0);
    const int rows = nt * 128;
    if (tid == 0) {
      tc::mbar_arrive_expect_tx(&t.bars[1], b_chunk);
      tc::bulk_g2s(sB, mx.phi_img, b_chunk, &t.bars[1]);
      if (staged) {
        for (int c = 0; c < 2 && c < chunks; ++c) {
          tc::mbar_arrive_expect_tx(&t.bars[5 + c], ph_bytes);
          tc::bulk_g2s(s_ph + c * ph_floats, mx.phi32c + (size_t)c * ph_floats, ph_bytes, &t.bars[5 + c]);
        }
      }
    }
    t.pend[1] = true;
    if (staged) {
      t.pend[5] = true;
      if (chunks > 1) t.pend[6] = true;
    }
    // A operand of chunk c: rows (ab, i) of this pass, nodes c kc .. c kc + kc - 1, both BF16 terms, into dst;
    // warps 1..7 (every thread waits for the staged chunk, so that the barrier phases stay uniform)
    auto build = [&](int c, uint8_t* dst) {
      const int q0 = c * mx.kc;
      if (staged && !tc_wait(t, 5 + (c & 1))) *s_abort = 1;
      const float* phc = staged ? s_ph + (c & 1) * ph_floats : nullptr;
      if (warp == 0) return;
#pragma unroll UNROLL
      for (int item = tid - 32; item < rows * groups; item += NT - 32) {
        const int rl = item >> gshift, g = item & (groups - 1);
        const int R = t0 * 128 + rl;
        uint32_t hw[4] = {0u, 0u, 0u, 0u}, lw[4] = {0u, 0u, 0u, 0u};
        if (R < BN) {
          const int ab = (int)__umulhi((uint32_t)R, inv_n), i = R - ab * N;   // R / N, R mod N
          const float* wj = s_wJf + ab * Q + q0 + g * 8;
          const int qe = Qc - q0 - g * 8;                 // entries of this group inside the rule
          float pv[8], wv[8];
          if (wj_vec) {
            const float4 v0 = reinterpret_cast<const float4*>(wj)[0], v1 = reinterpret_cast<const float4*>(wj)[1];
            wv[0] = v0.x; wv[1] = v0.y; wv[2] = v0.z; wv[3] = v0.w;
            wv[4] = v1.x; wv[5] = v1.y; wv[6] = v1.z; wv[7] = v1.w;
          } else {
#pragma unroll
            for (int e = 0; e < 8; ++e) wv[e] = e < qe ? wj[e] : 0.f;
          }
          if (staged) {
            // rows of kcp = kc + 4 floats: the two 16-byte loads of a quarter warp hit 32 distinct banks
            const float4* p4 = reinterpret_cast<const float4*>(phc + i * kcp + g * 8);
            const float4 u0 = p4[0], u1 = p4[1];
            pv[0] = u0.x; pv[1] = u0.y; pv[2] = u0.z; pv[3] = u0.w;
            pv[4] = u1.x; pv[5] = u1.y; pv[6] = u1.z; pv[7] = u1.w;
          } else {
            const float* ph = mx.phiT32 + (size_t)i * Q + q0 + g * 8;
#pragma unroll
            for (int e = 0; e < 8; ++e) pv[e] = e < qe ? ph[e] : 0.f;
          }
#pragma unroll
          for (int e = 0; e < 8; e += 2) {
            const float x0 = e < qe ? wv[e] * pv[e] : 0.f;
            const float x1 = e + 1 < qe ? wv[e + 1] * pv[e + 1] : 0.f;
            const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
            const float2 hf = __bfloat1622float2(h);
            const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
            hw[e / 2] = *reinterpret_cast<const uint32_t*>(&h);
            lw[e / 2] = *reinterpret_cast<const uint32_t*>(&l);
          }
        }
        const uint32_t off = tc::kmajor_offset(rl, g * 8, sbo);
        *reinterpret_cast<uint4*>(dst + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4*>(dst + a_img + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
      }
    };
    // With two A buffers warps 1..7 build chunk c + 1 while the MMAs of chunk c run; with one, after them.
    build(0, sA);
    tc::fence_proxy_async();
    __syncthreads();
    for (int c = 0; c < chunks; ++c) {
      const int buf = c & 1;
      uint8_t* a_cur = sA + (two_a ? buf : 0) * a_buf;
      if (c + 1 < chunks) {
        // the other B buffer was last read by the MMAs of chunk c-1, which have completed
        if (tid == 0) {
          tc::mbar_arrive_expect_tx(&t.bars[1 + (buf ^ 1)], b_chunk);
          tc::bulk_g2s(sB + (buf ^ 1) * b_chunk, mx.phi_img + (size_t)(c + 1) * b_chunk, b_chunk,
                       &t.bars[1 + (buf ^ 1)]);
        }
        t.pend[1 + (buf ^ 1)] = true;
      }
      if (staged && c + 2 < chunks) {
        // staged buffer c & 1 was last read by the build of chunk c, which has completed
        if (tid == 0) {
          tc::mbar_arrive_expect_tx(&t.bars[5 + buf], ph_bytes);
          tc::bulk_g2s(s_ph + buf * ph_floats, mx.phi32c + (size_t)(c + 2) * ph_floats, ph_bytes, &t.bars[5 + buf]);
        }
        t.pend[5 + buf] = true;
      }
      const bool got_b = tc_wait(t, 1 + buf);
      if (!got_b) *s_abort = 1;
      if (tid == 0 && got_b) {
        tc::fence_after_sync();
        const uint32_t sa = tc::smem_u32(a_cur), sb = tc::smem_u32(sB + buf * b_chunk);
        for (int tl = 0; tl < nt; ++tl) {
          const uint32_t d = t.tmem + (uint32_t)(tl * acc_cols);
          const uint32_t ta = sa + (uint32_t)tl * 16u * sbo;   // 128 rows = 16 row groups
          for (int ks = 0; ks < mx.kc / 16; ++ks) {
            const uint32_t kofs = (uint32_t)ks * 256u;
            const uint64_t ah = tc::smem_desc(ta + kofs, sbo), al = tc::smem_desc(ta + a_img + kofs, sbo);
            const uint64_t bh = tc::smem_desc(sb + kofs, sbo);
            const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
            if (stack) {
              tc::mma_bf16(d, ah, bh, idesc2, acc);          // [A_hi B_hi | A_hi B_lo]
              tc::mma_bf16(d, al, bh, idesc, 1u);            // + A_lo B_hi into the first half
            } else {
              const uint64_t bl = tc::smem_desc(sb + b_img + kofs, sbo);
              tc::mma_bf16(d, ah, bh, idesc, acc);
              tc::mma_bf16(d, ah, bl, idesc, 1u);
              tc::mma_bf16(d, al, bh, idesc, 1u);
            }
          }
        }
        tc::mma_commit(&t.bars[0]);
      }
      if (got_b) t.pend[0] = true;
      // the other A buffer was last read by the MMAs of chunk c-1, which have completed
      if (two_a && c + 1 < chunks) build(c + 1, sA + (buf ^ 1) * a_buf);
      if (!tc_wait(t, 0)) *s_abort = 1;
      if (!two_a && c + 1 < chunks) build(c + 1, sA);
      tc::fence_proxy_async();
      tc::fence_after_sync();
      __syncthreads();
      if (*s_abort) return false;
    }
    // accumulators -> packed FP64 H. Warp w reads tensor-memory lanes 32 (w % 4) .. + 31 and one
    // half of the columns, eight at a time (with the stacked operand both accumulators before one wait).
    const int lq = warp & 3, half = warp >> 2;
    const int hcols = n_pad / 2;
    for (int tl = 0; tl < nt; ++tl) {
      const int R = (t0 + tl) * 128 + lq * 32 + lane;
      const bool valid = R < BN;
      const int ab = valid ? R / N : 0, i = valid ? R - ab * N : 0;
      int aa, bb;
      unpack_ab<M>(ab, aa, bb);
      // the value H_ab[i][j] goes to packed row i M + a, column j M + b (j < i, or j <= i when a = b) and,
      // for a < b, also to row i M + b, column j M + a (j <= i)
      const size_t o1 = rowoff(i * M + aa) + bb, o2 = rowoff(i * M + bb) + aa;
      const int jmax1 = aa == bb ? i : i - 1;
      const uint32_t tbase = t.tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(tl * acc_cols);
      for (int cg = 0; cg < hcols; cg += 8) {
        const int col0 = half * hcols + cg;
        uint32_t r[8], r2[8];
        tc::tmem_ld_x8(tbase + (uint32_t)col0, r);
        if (stack) tc::tmem_ld_x8(tbase + (uint32_t)(n_pad + col0), r2);
        tc::tmem_wait_ld();
        if (valid) {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int j = col0 + e;
            if (j <= i) {
              const float f = stack ? __uint_as_float(r[e]) + __uint_as_float(r2[e]) : __uint_as_float(r[e]);
              const T v = widen<T>(f);
              if (j <= jmax1) s_H[o1 + (size_t)j * M] = v;
              if (aa != bb) s_H[o2 + (size_t)j * M] = v;
            }
          }
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
  }
  return true;
}

// ------------------------------------------------------------------------------------------------
// (c), split variant: the right-looking factorisation of cholesky_aug with outer panels of SNB = 16
// columns, whose trailing updates A22 -= L21 L21^T run on the tensor cores as exact integer products.
//
// Each row r of a finished panel (16 entries of L21; the gradient row n included) is written as
// 2^e_r sum_{i=1..7} d_i 2^(-8i): e_r is the exponent of the row's largest entry and the integer digits
// d_i, |d_i| <= 255, are the base-256 digits of the entries' binary expansions truncated to 56 bits
// (the error-free splitting of Ozaki, Ogita and Oishi, 2012, with one scale per row). A digit is exact in
// BF16 and a product of two digits exact in FP32. For every output entry the seven diagonals
// D_t = sum_{i+j=t} sum_k d_i[r][k] d_j[c][k], t = 2..8, are accumulated by tcgen05.mma in seven FP32
// accumulators in tensor memory; a diagonal sums at most 7 x 16 products below 2^16, so it stays below
// 2^24 and is exact. The diagonals are combined exactly in a 64-bit integer, 2^56 S = sum_t D_t 2^(56-8t)
// (the t = 8 term truncated), converted to FP64 and subtracted as A22 -= 2^(e_r + e_c - 56) (2^56 S).
// The roundings are the 56-bit truncation of the digits (relative to the row's largest entry), the
// conversion of 2^56 S and the final FMA: FP64-level accuracy, with the FP64 work of a trailing entry cut
// from 16 FMAs per panel to one conversion and one FMA. The panel itself (two blocks of NB = 8 columns)
// is factorised in FP64 by panel_diag / panel_trsm as in cholesky_aug, one panel ahead of the trailing update.
// Digit slices: SDIG arrays of s_rows x 16 BF16 in the K-major core-matrix layout (8-row groups SSBO
// bytes apart), rows counted from the first trailing row s1; rows beyond the trailing block hold stale
// data that only ever feeds output rows and columns that are not read back.
// ------------------------------------------------------------------------------------------------
constexpr int SNB = 16;                 // outer panel width = MMA K
constexpr int SDIG = 7;                 // base-256 digits per entry (56 bits)
constexpr int SBLK = 32;                // output columns per MMA (N)
constexpr uint32_t SSBO = 256;          // tc::kmajor_sbo(16)
constexpr int SPLIT_BUF_COLS = SPLIT_TMEM_COLS_ONE;   // tensor-memory columns of one accumulator set
static_assert(SDIG * SBLK <= SPLIT_BUF_COLS, "the seven diagonals of a unit must fit one accumulator set");

struct SplitSmem {
  uint8_t* slices;   // SDIG x rows x 16 BF16
  int* rexp;         // [rows] biased exponent field of each row's largest entry
  int rows;          // rows per slice (multiple of 32, >= 128)
  int nbuf;          // accumulator sets in tensor memory (1, or 2 to overlap MMAs with the combine)
};

// Digit slices and row exponents of rows s1..n of the panel columns kb..kb+kw-1 (kw <= 16; the other
// columns get zero digits). Two threads per row, eight columns each.
static __device__ void split_panel(const double* A, int n, int kb, int kw, int s1, const SplitSmem& sp) {
  const int R = n + 1 - s1;
  const uint32_t slice_bytes = (uint32_t)sp.rows * 32u;
  for (int base = 0; base < 2 * R; base += NT) {
    const int item = base + threadIdx.x;
    const bool valid = item < 2 * R;
    const int rs = item >> 1, half = item & 1;
    long long bits[8];
    int emax = 0;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = half * 8 + e;
      bits[e] = (valid && k < kw) ? __double_as_longlong(A[rowoff(s1 + rs) + kb + k]) : 0ll;
      emax = max(emax, (int)((bits[e] >> 52) & 0x7FF));
    }
    emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, 1));
    if (valid) {
      // Digits as BF16 from 32-bit words: the 56-bit X is split into its high 24 and low 32 bits, a digit
      // 0 <= d <= 255 is made exact in FP32 as (2^23 + d) - 2^23 and its BF16 is the float's high half
      // (d has at most 8 significant bits); two columns' halves are packed with one byte permute.
      uint32_t w[SDIG][4];
#pragma unroll
      for (int pr = 0; pr < 4; ++pr) {
        uint32_t xh[2], xl[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const long long b = bits[2 * pr + h];
          const int E = (int)((b >> 52) & 0x7FF);
          unsigned long long X = 0ull;
          if (E != 0) {
            const unsigned long long mant = ((unsigned long long)b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
            const int sh = E - emax + 3;                  // <= 3: X < 2^56
            X = sh >= 0 ? (mant << sh) : (sh > -64 ? (mant >> -sh) : 0ull);
          }
          xh[h] = (uint32_t)(X >> 32);
          xl[h] = (uint32_t)X;
        }
        const uint32_t sgn = (bits[2 * pr] < 0 ? 0x8000u : 0u) | (bits[2 * pr + 1] < 0 ? 0x80000000u : 0u);
#pragma unroll
        for (int i = 0; i < SDIG; ++i) {
          uint32_t d0, d1;                                // digit i: bits 48 - 8 i .. 55 - 8 i of X
          if (i < 3) {
            d0 = (xh[0] >> (16 - 8 * i)) & 0xFFu;
            d1 = (xh[1] >> (16 - 8 * i)) & 0xFFu;
          } else {
            d0 = (xl[0] >> (48 - 8 * i)) & 0xFFu;
            d1 = (xl[1] >> (48 - 8 * i)) & 0xFFu;
          }
          const float f0 = __uint_as_float(0x4B000000u | d0) - 8388608.0f;
          const float f1 = __uint_as_float(0x4B000000u | d1) - 8388608.0f;
          w[i][pr] = __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632) | sgn;
        }
      }
      const uint32_t off = (uint32_t)(rs >> 3) * SSBO + (uint32_t)half * 128u + (uint32_t)(rs & 7) * 16u;
#pragma unroll
      for (int i = 0; i < SDIG; ++i)
        *reinterpret_cast<uint4*>(sp.slices + i * slice_bytes + off) = make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
      if (half == 0) sp.rexp[rs] = emax;
    }
  }
}

// Work unit u of a trailing update with R rows (row slots 0..R-1; column slots 0..R-2): a 128-row MMA
// tile starting at slot ta that owns the output rows [lo, hi), and a block of SBLK columns from cb.
// Units are ordered with the first column block of every tile first (they hold the next panel's columns).
__device__ __forceinline__ bool split_unit(int u, int R, int& ta, int& lo, int& hi, int& cb) {
  const int R8 = (R + 7) & ~7;
  const int ntl = (R + 127) / 128;
  int k = -1;
  if (u < ntl) {
    k = u;
    cb = 0;
  } else {
    u -= ntl;
    for (int l = 0; l < R && k < 0; l += 128) {
      const int nb = (min(min(R, l + 128), R - 1) + SBLK - 1) / SBLK - 1;   // blocks after the first
      if (u < nb) {
        k = l / 128;
        cb = (u + 1) * SBLK;
      } else {
        u -= nb;
      }
    }
    if (k < 0) return false;
  }
  lo = 128 * k;
  hi = min(R, lo + 128);
  ta = min(lo, max(0, R8 - 128));
  return true;
}

__device__ __forceinline__ int split_units(int R) {
  int U = 0;
  for (int l = 0; l < R; l += 128) U += (min(min(R, l + 128), R - 1) + SBLK - 1) / SBLK;
  return U;
}

// One thread issues the 28 digit-pair MMAs of a unit into accumulator set d (D_t at column (t-2) SBLK).
__device__ __forceinline__ void split_mma(uint32_t d, uint32_t sl, uint32_t slice_bytes, int ta, int cb) {
  const uint32_t idesc = tc::idesc_bf16_f32(128, SBLK);
#pragma unroll
  for (int t = 2; t <= SDIG + 1; ++t) {
#pragma unroll
    for (int i = 1; i < t; ++i) {
      const int j = t - i;
      const uint64_t ad = tc::smem_desc(sl + (uint32_t)(i - 1) * slice_bytes + (uint32_t)(ta >> 3) * SSBO, SSBO);
      const uint64_t bd = tc::smem_desc(sl + (uint32_t)(j - 1) * slice_bytes + (uint32_t)(cb >> 3) * SSBO, SSBO);
      tc::mma_bf16(d + (uint32_t)((t - 2) * SBLK), ad, bd, idesc, i > 1 ? 1u : 0u);
    }
  }
}

__device__ __forceinline__ long long split_digit_sum(const uint32_t (&v)[SDIG][8], int e) {
  long long acc = 0;
#pragma unroll
  for (int t = 0; t < SDIG; ++t) {
    const long long dt = (long long)__float2int_rz(__uint_as_float(v[t][e]));
    const int sh = 40 - 8 * t;                       // D_(t+2) 2^(56 - 8 (t+2))
    acc += sh >= 0 ? (dt << sh) : (dt >> -sh);
  }
  return acc;
}

// A[s1 + rs][s1 + cs] -= L21 L21^T for the unit's entries (rows [lo, hi), lower triangle, columns < n).
// The calling warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (tile rows) and the block's columns
// [8 g0, 8 g1).
static __device__ void split_combine(double* A, int s1, int R, int lo, int hi, int ta, int cb, uint32_t d, const int* rexp,
                                     int g0, int g1) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lq = warp & 3;
  const int rs = ta + lq * 32 + lane;
  const bool row_ok = rs >= lo && rs < hi;
  const int Er = row_ok ? rexp[rs] : 0;
  double* Arow = A + rowoff(row_ok ? s1 + rs : 0) + s1;
  for (int cg = g0; cg < g1; ++cg) {
    const int c0 = cg * 8;
    uint32_t v[SDIG][8];
#pragma unroll
    for (int t = 0; t < SDIG; ++t)
      tc::tmem_ld_x8(d + ((uint32_t)(lq * 32) << 16) + (uint32_t)(t * SBLK + c0), v[t]);
    tc::tmem_wait_ld();
    if (row_ok) {
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int cs = cb + c0 + e;
        if (cs <= rs && cs < R - 1) {
          const long long acc = split_digit_sum(v, e);
          const int ex = Er + rexp[cs] - 1077;        // biased exponent of 2^(e_r + e_c - 56)
          if (acc != 0 && ex >= 1) Arow[cs] = fma(-(double)acc, __longlong_as_double((long long)ex << 52), Arow[cs]);
        }
      }
    }
  }
}

// The 16-column panel kb..kb+kw-1 (rows kb..n, already updated by every earlier panel) is factorised in
// FP64 in up to four phases, each a block-wide step between two barriers: 0 the diagonal block of its
// first NB columns (one warp, panel_diag), 1 their rows below (panel_trsm), 2 the second block's columns
// updated by the first, with warp 0 taking the rows of the second diagonal block and factorising that
// block right after (the other threads update the rows below it meanwhile), 3 the second block's rows
// below. Threads t0, t0 + stride, ... share the row work (t0 < 32: warp 0). The first block's columns go
// to the panel buffer P, the second block's to the buffer after it (P + (n + 1) PSTR), so that the rows
// below still read the first block's values while warp 0 factorises the second diagonal block.
__device__ __forceinline__ int panel_phases(int kw) { return kw > NB ? 4 : 2; }

static __device__ void panel_phase(int ph, double* A, int n, int kb, int kw, double* P, double* s_dinv, int* s_flag,
                                   int t0, int stride) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k0 = min(NB, kw), s0 = kb + NB, k1 = kw - NB;
  double* P1 = P + (size_t)(n + 1) * PSTR;
  if (ph == 0) {
    if (warp == 0) panel_diag(A, kb, k0, P, s_dinv, s_flag);
  } else if (ph == 1) {
    panel_trsm(A, n, kb, k0, P, s_dinv, t0, stride);
  } else if (ph == 2) {
    if (warp == 0) {
      // rows s0 .. s0 + k1 - 1 (lane i: row s0 + i), then their diagonal block
      if (lane < k1) {
        const int r = s0 + lane;
        for (int c = s0; c <= r; ++c) {
          double acc = 0.0;
#pragma unroll
          for (int k = 0; k < NB; ++k) acc = fma(P[r * PSTR + k], P[c * PSTR + k], acc);
          A[rowoff(r) + c] -= acc;
        }
      }
      __syncwarp();
      panel_diag(A, s0, k1, P1, s_dinv, s_flag);
    } else {
      const int r0 = s0 + k1, rows = n + 1 - r0;
      for (int item = t0 - 32; item < rows * k1; item += stride - 32) {
        const int r = r0 + item / k1, c = s0 + item % k1;
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < NB; ++k) acc = fma(P[r * PSTR + k], P[c * PSTR + k], acc);
        A[rowoff(r) + c] -= acc;
      }
    }
  } else {
    panel_trsm(A, n, s0, k1, P1, s_dinv, t0, stride);
  }
}

// Split factorisation of the packed (n+1) x (n+1) augmented matrix (rows 0..n-1: H, row n: g), with
// the forward substitution folded in as in cholesky_aug. Returns false on a bad pivot (*s_flag set) or
// when a bounded tensor-core wait ran out (*s_abort set).
// One panel of look-ahead: the trailing units of a panel start with the first column block of every row
// tile, which holds the next panel's columns. Once the unit with the next diagonal block (and for the
// later phases, every first column block) is combined, each unit iteration also advances one phase of
// the next panel on warps 0..3, while warps 4..7 (one per tensor-memory lane quadrant) combine that unit
// alone; the other units are combined by all eight warps (two per quadrant, half of the columns each).
// The phases touch only the next panel's 16 columns, the panel buffer and the pivots; the units combined
// beside them only columns 32 and more to the right, so the two never meet. Phases left over when the
// units run out follow on all warps.
static __device__ bool cholesky_split(double* A, int n, double* s_P, double* s_dinv, int* s_flag, const SplitSmem& sp,
                                      TcState& t, int* s_abort) {
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t sl = tc::smem_u32(sp.slices);
  const uint32_t slice_bytes = (uint32_t)sp.rows * 32u;
  if (tid == 0) *s_flag = 0;
  __syncthreads();
  {
    const int kw0 = min(SNB, n);
    for (int ph = 0; ph < panel_phases(kw0); ++ph) {
      panel_phase(ph, A, n, 0, kw0, s_P, s_dinv, s_flag, tid, NT);
      __syncthreads();
      if (*s_flag) return false;
    }
  }
  for (int kb = 0; kb < n; kb += SNB) {
    // this panel is factorised (above, or by the look-ahead of the previous panel)
    const int kw = min(SNB, n - kb);
    const int s1 = kb + kw;
    if (s1 >= n) break;                              // only the gradient row is below: nothing to update
    const int R = n + 1 - s1;
    const int kw1 = min(SNB, n - s1);                // the next panel
    const int nph = panel_phases(kw1);
    const int ntl = (R + 127) / 128;                 // units 0 .. ntl-1: the first column block of each tile
    int ph = 0;
    split_panel(A, n, kb, kw, s1, sp);
    tc::fence_proxy_async();
    __syncthreads();
    const int U = split_units(R);
    auto issue = [&](int u) {
      const int b = u % sp.nbuf;
      if (tid == 0) {
        int ta, lo, hi, cb;
        split_unit(u, R, ta, lo, hi, cb);
        tc::fence_after_sync();
        split_mma(t.tmem + (uint32_t)(b * SPLIT_BUF_COLS), sl, slice_bytes, ta, cb);
        tc::mma_commit(&t.bars[3 + b]);
      }
      t.pend[3 + b] = true;
    };
    issue(0);
    for (int u = 0; u < U; ++u) {
      const int b = u % sp.nbuf;
      if (sp.nbuf == 2 && u + 1 < U) issue(u + 1);
      if (!tc_wait(t, 3 + b)) *s_abort = 1;
      tc::fence_after_sync();
      int ta, lo, hi, cb;
      split_unit(u, R, ta, lo, hi, cb);
      const uint32_t d = t.tmem + (uint32_t)(b * SPLIT_BUF_COLS);
      const bool ahead = ph < nph && !*s_flag && u >= (ph == 0 ? 1 : ntl);
      if (ahead) {
        if (warp >= 4) split_combine(A, s1, R, lo, hi, ta, cb, d, sp.rexp, 0, 4);
        else panel_phase(ph, A, n, s1, kw1, s_P, s_dinv, s_flag, tid, 128);
        ++ph;
      } else {
        split_combine(A, s1, R, lo, hi, ta, cb, d, sp.rexp, 2 * (warp >> 2), 2 * (warp >> 2) + 2);
      }
      tc::fence_before_sync();
      __syncthreads();
      if (*s_abort) return false;
      if (sp.nbuf == 1 && u + 1 < U) issue(u + 1);
    }
    for (; ph < nph && !*s_flag; ++ph) {
      panel_phase(ph, A, n, s1, kw1, s_P, s_dinv, s_flag, tid, NT);
      __syncthreads();
    }
    if (*s_flag) return false;
  }
  return true;
}

// ------------------------------------------------------------------------------------------------
// 1-D Lax-Friedrichs update folded into the Newton launch (Algorithm 1, the moment update; App. A).
// With nu = dx / (2 dt) the update of cell j,
//   u_hat_j = sum_k w_k [u_j - dt/dx (g(u_j, u_r) - g(u_l, u_j))] phi(xi_k),
// reduces to A_j - (dt/dx) B_j with A_j = sum_k w_k (u_l + u_r)/2 phi and B_j = sum_k w_k (f(u_r) -
// f(u_l))/2 phi: the centre value cancels and neither term needs dt, which is known only when every
// cell is solved. Cell k, once its nodal states are final, counts itself towards each cell whose
// neighbour it is; the CTA that completes a count forms that cell's A and B. Fixed (Dirichlet) ghosts
// are final from the start and are not counted; a cell with two of them is formed by its own CTA.
// Scratch: s_ia, s_ib [M][Q] integrands, s_part [2][NWARPS][NM] partial sums; all threads call.
// ------------------------------------------------------------------------------------------------
template <int PHYS, int M>
__device__ void lf_fold(const NewtonArgs& a, int k, double* s_ia, double* s_ib, double* s_part, int* s_ready) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nx = a.nx, Q = a.tab.Q, N = a.tab.N, NM = N * M;
  __threadfence();                                   // this CTA's nodal states of k, before the counts
  __syncthreads();
  if (tid == 0) {
    int n = 0;
    const int cand[5] = {k - 1, k + 1, k, 1, nx};
    for (int ci = 0; ci < 5; ++ci) {
      const int j = cand[ci];
      bool seen = j < 1 || j > nx;
      for (int cj = 0; cj < ci; ++cj) seen = seen || cand[cj] == j;
      if (seen) continue;
      const int jl = neighbour(j, nx, -1, a.bc_left), jr = neighbour(j, nx, +1, a.bc_right);
      const bool il = jl >= 1 && jl <= nx, ir = jr >= 1 && jr <= nx && jr != jl;
      const int target = (il ? 1 : 0) + (ir ? 1 : 0);
      if (target == 0) {
        if (j == k) s_ready[n++] = j;
      } else if (jl == k || jr == k) {
        if (atomicAdd(&a.lf_cnt[j], 1) == target - 1) s_ready[n++] = j;
      }
    }
    __threadfence();                                 // the other CTAs' nodal states, after the counts
    s_ready[3] = n;
  }
  __syncthreads();
  const int n_ready = s_ready[3];
  const double* __restrict__ w = a.tab.w;
  const double* __restrict__ Phi = a.tab.Phi;
  const int MQ = M * Q;
  const int qw = (Q + NWARPS - 1) / NWARPS;
  const int q_lo = min(Q, warp * qw), q_hi = min(Q, q_lo + qw);
  for (int t = 0; t < n_ready; ++t) {
    const int j = s_ready[t];
    const double* ul_g = a.unode + (size_t)neighbour(j, nx, -1, a.bc_left) * MQ;
    const double* ur_g = a.unode + (size_t)neighbour(j, nx, +1, a.bc_right) * MQ;
    for (int q = tid; q < Q; q += NT) {
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
    __syncthreads();
    // projections: warp k sums the nodes [k qw, (k+1) qw) for every entry; partials added in warp order
    for (int rr = lane; rr < NM; rr += 32) {
      const int i = rr / M, c = rr - i * M;
      double sa = 0.0, sb = 0.0;
      for (int q = q_lo; q < q_hi; ++q) {
        const double ph = Phi[(size_t)q * N + i];
        sa = fma(ph, s_ia[c * Q + q], sa);
        sb = fma(ph, s_ib[c * Q + q], sb);
      }
      s_part[warp * NM + rr] = sa;
      s_part[(NWARPS + warp) * NM + rr] = sb;
    }
    __syncthreads();
    for (int rr = tid; rr < NM; rr += NT) {
      double va = 0.0, vb = 0.0;
#pragma unroll
      for (int kw = 0; kw < NWARPS; ++kw) {
        va += s_part[kw * NM + rr];
        vb += s_part[(NWARPS + kw) * NM + rr];
      }
      a.lf_a[(size_t)j * NM + rr] = va;
      a.lf_b[(size_t)j * NM + rr] = vb;
    }
    __syncthreads();
  }
}

// Duration of one tensor-core Hessian phase (entry of hessian_tc to its final block barrier, as seen by
// thread 0), added to the step counters: the in-phase tensor-pipe rate of row (b) is its tensor flops
// over this time.
__device__ __forceinline__ void hessian_timed(StepScalars* sc, uint64_t t0) {
  atomicAdd(&sc->hessian_ns, (unsigned long long)(tc::globaltimer() - t0));
  atomicAdd(&sc->hessian_count, 1ULL);
}

// The split variants run one CTA per SM (their systems fill the shared memory) and get its registers.
template <int ENT, int PHYS, int M, bool H_SMEM, bool MIXED, bool F32F, bool SPLIT>
__global__ void __launch_bounds__(NT, SPLIT ? 1 : 2) k_newton(NewtonArgs a) {
  constexpr bool TC = MIXED || SPLIT;   // tensor memory and barriers in use
  constexpr int B = packed_count(M);
  extern __shared__ __align__(128) double smem[];
  __shared__ int s_work;
  __shared__ int s_abort;
  __shared__ int s_flag;
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_bars[TC_BARS];
  __shared__ int s_lf_ready[4];
  // shared arrays are sized for the table's N (the finest level); a cell may use fewer moments
  const int NX = a.tab.N, Q = a.tab.Q, NMX = NX * M;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double* s_lam = smem;
  double* s_uh = s_lam + NMX;
  double* s_g = s_uh + NMX;
  double* s_d = s_g + NMX;
  double* s_Lam = s_d + NMX;      // [M][Q]
  double* s_dLam = s_Lam + M * Q; // [M][Q]
  double* s_u = s_dLam + M * Q;   // [M][Q]
  double* s_wJ = s_u + M * Q;     // [B][Q]  (float [B][Q] on the mixed path, half the space)
  double* s_red = s_wJ + (MIXED ? (B * Q + 1) / 2 : B * Q);   // NWARPS * 8
  double* s_wu = s_red + NWARPS * 8;  // [M][Q] w_k u_k
  double* s_dinv = s_wu + M * Q;      // [NM] reciprocal pivots
  double* s_P = s_dinv + NMX;         // [2][(NM + 1) * PSTR] Cholesky panels (current, next)
  uint8_t* sbytes = reinterpret_cast<uint8_t*>(smem);
  double* s_H = H_SMEM ? reinterpret_cast<double*>(sbytes + a.off_h) : (a.hwork + (size_t)blockIdx.x * a.hwork_stride);
  uint8_t* sA = sbytes + a.off_a;
  uint8_t* sB = sbytes + a.off_b;
  float* s_ph = (MIXED && a.mx.off_ph) ? reinterpret_cast<float*>(sbytes + a.mx.off_ph) : nullptr;
  const double* __restrict__ PhiT = a.tab.PhiT;
  const double* __restrict__ Phi = a.tab.Phi;
  const double* __restrict__ w = a.tab.w;

  TcState tcs;
  tcs.bars = s_bars;
  tcs.tmem = 0;
  for (int k = 0; k < TC_BARS; ++k) {
    tcs.ph[k] = 0u;
    tcs.pend[k] = false;
  }
  SplitSmem ssp;
  ssp.slices = sbytes + a.off_s;
  ssp.rexp = reinterpret_cast<int*>(sbytes + a.off_s + (size_t)SDIG * a.s_rows * 32);
  ssp.rows = a.s_rows;
  ssp.nbuf = a.s_nbuf;
  if (TC) {
    if (tid == 0) {
      s_abort = 0;
      for (int k = 0; k < TC_BARS; ++k) tc::mbar_init(&s_bars[k], 1);
      tc::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(&s_tmem, (uint32_t)a.mx.tmem_cols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    tcs.tmem = s_tmem;
  }

  const int n_work = a.count_dev ? *a.count_dev : a.n_work;
  int* queue = a.queue ? a.queue : &a.sc->work_counter;
  bool stop = false;
  while (!stop) {
    if (tid == 0) s_work = atomicAdd(queue, 1);
    __syncthreads();
    const int wk = s_work;
    if (wk >= n_work) break;
    const int cell = a.cell_list ? a.cell_list[wk] : work_cell(wk, a.nx, a.gy);
    const int N = a.level ? a.lev_n[a.level[cell]] : NX;     // moments of this cell's level
    const int NM = N * M;
    // this cell's quadrature: its level's rule (the first Qc of the table's nodes) or the shared rule
    const int lev_c = a.level ? a.level[cell] : 0;
    const int Qc = a.lev_w ? a.lev_q[lev_c] : Q;
    const double* __restrict__ wc = a.lev_w ? a.lev_w + (size_t)lev_c * Q : w;
    double* lam_g = a.lam + (size_t)cell * NMX;
    const double* uh_g = a.uhat + (size_t)cell * NMX;
    for (int r = tid; r < NM; r += NT) {
      s_lam[r] = lam_g[r];
      s_uh[r] = uh_g[r];
    }
    __syncthreads();

    // Convergence check from the moment image. While the duals are bit for bit those the cell's last
    // successful solve ended at, the gradient at the start of this solve is S - u_hat (Eq. gradient)
    // with exactly the arithmetic of a fresh evaluation (same nodes, same sums), so a cell whose new
    // moments already meet Eq. tauCrit needs no reconstruction and no closures; its nodal states and
    // wave speed are those its last solve left for the same duals.
    // The images are kept by every solve that moves the duals (One-Shot steps included); a Hessian dump
    // leaves them out and only invalidates.
    const bool dump = a.h_dump != nullptr || a.f_dump != nullptr;   // Hessian / factor dump: no update
    const bool img_rd = a.img != nullptr && !a.one_step && !dump;
    const bool img_wr = a.img != nullptr && !dump;
    if (img_rd) {
      bool same = a.img_valid[cell] == lev_c + 1;     // the image belongs to this level
      if (same) {
        const double* Sc = a.img + (size_t)cell * NMX;
        const double* Lc = a.img_lam + (size_t)cell * NMX;
        for (int r = tid; r < NM; r += NT) {
          same = same && __double_as_longlong(Lc[r]) == __double_as_longlong(s_lam[r]);
          s_g[r] = Sc[r] - s_uh[r];
        }
      }
      if (__syncthreads_and(same)) {
        const double res = grad_residual<M>(s_g, N, s_red);
        if (res < a.tau) {                           // false for NaN
          if (tid == 0) {
            a.iters[cell] = 0;
            a.status[cell] = ST_OK;
            atomicAdd(&a.sc->cached_checks, 1ULL);
            if (a.track_speed) atomic_max_pos(&a.sc->smax_bits, a.img_smax[cell]);
          }
          __syncthreads();
          if constexpr (PHYS != PHYS_EULER2D)
            if (a.lf_a) lf_fold<PHYS, M>(a, cell, s_Lam, s_dLam, s_P, s_lf_ready);
          continue;
        }
      }
    }
    if (a.img != nullptr && tid == 0) a.img_valid[cell] = 0;   // this solve rewrites the cell's states

    int it = 0, st = ST_OK;
    // frozen Hessians (hessian_reuse > 0): the Cholesky factor of an earlier iterate is kept and reused
    // while the Newton steps it gives converge fast enough
    bool have_factor = false;
    int nfact = 0;
    double res_prev = 0.0, alpha_prev = 0.0;
    if (a.hessian_reuse == 2 && a.factor_valid[cell]) {
      const double* fs = a.factor_store + (size_t)cell * a.factor_stride;
      const size_t nph = (size_t)NM * (NM + 1) / 2;
      for (size_t r = tid; r < nph; r += NT) s_H[r] = fs[r];
      for (int r = tid; r < NM; r += NT) s_dinv[r] = fs[nph + r];
      have_factor = true;
    }
    for (;;) {
      // (a1) reconstruction
      for (int q = tid; q < Qc; q += NT) {
        double acc[M];
#pragma unroll
        for (int c = 0; c < M; ++c) acc[c] = 0.0;
#pragma unroll 4
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
      for (int q = tid; q < Qc; q += NT) {
        double L[M], u[M], J[B], ss;
#pragma unroll
        for (int c = 0; c < M; ++c) L[c] = s_Lam[c * Q + q];
        const bool ok = Closure<ENT, M>::template eval<true>(L, a.ent, u, J, ss);
        const double wq = wc[q];
#pragma unroll
        for (int c = 0; c < M; ++c) {
          s_u[c * Q + q] = u[c];
          s_wu[c * Q + q] = wq * u[c];
        }
        if (MIXED) {
          float* s_wJf = reinterpret_cast<float*>(s_wJ);
#pragma unroll
          for (int b = 0; b < B; ++b) s_wJf[b * Q + q] = (float)(wq * J[b]);
        } else {
#pragma unroll
          for (int b = 0; b < B; ++b) s_wJ[b * Q + q] = wq * J[b];
        }
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
      // (a3) gradient g_(i,c) = sum_k w_k u_c(xi_k) phi_i(xi_k) - u_hat_(i,c), one thread per entry
      for (int r = tid; r < NM; r += NT) {
        const int i = r / M, c = r - i * M;
        const double* wu = s_wu + c * Q;
        // four independent partial sums: the node sum is a dependent chain otherwise
        double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0, acc3 = 0.0;
        int q = 0;
        for (; q + 4 <= Qc; q += 4) {
          acc0 = fma(Phi[(size_t)q * NX + i], wu[q], acc0);
          acc1 = fma(Phi[(size_t)(q + 1) * NX + i], wu[q + 1], acc1);
          acc2 = fma(Phi[(size_t)(q + 2) * NX + i], wu[q + 2], acc2);
          acc3 = fma(Phi[(size_t)(q + 3) * NX + i], wu[q + 3], acc3);
        }
        for (; q < Qc; ++q) acc0 = fma(Phi[(size_t)q * NX + i], wu[q], acc0);
        const double S = (acc0 + acc1) + (acc2 + acc3);
        s_g[r] = S - s_uh[r];
        if (img_wr) a.img[(size_t)cell * NMX + r] = S;
      }
      __syncthreads();
      const double res = grad_residual<M>(s_g, N, s_red);

      if (red[2] > 0.0) { st = ST_INFEASIBLE; break; }
      if (!isfinite(res)) { st = ST_NONFINITE; break; }
      if (!dump) {
        if (a.one_step) {
          if (it >= 1) break;
        } else {
          if (res < a.tau) break;
          if (it >= a.max_newton) { st = ST_NOCONV; break; }
        }
      }

      const bool reuse = have_factor && a.hessian_reuse > 0 && !dump &&
                         (it == 0 ? a.hessian_reuse == 2 : (alpha_prev == 1.0 && res <= a.reuse_ratio * res_prev));
      res_prev = res;
      bool solved = false;
      if (F32F && !reuse && !dump) {
        // FP32 factorisation of the split-BF16 Hessian: the tensor-core accumulators are FP32 already;
        // the FP32 solve gives the Newton direction to about the Hessian's own accuracy. A failed
        // pivot falls through to the FP64 assembly and factorisation below.
        float* Hf = reinterpret_cast<float*>(s_H);
        float* Pf = reinterpret_cast<float*>(s_P);
        float* dinvf = reinterpret_cast<float*>(s_dinv);
        const uint64_t th0 = tid == 0 ? tc::globaltimer() : 0;
        if (!hessian_tc<M, float, SPLIT ? 2 : 1>(a, N, Qc, reinterpret_cast<const float*>(s_wJ), Hf, sA, sB, s_ph, tcs, &s_abort)) {
          if (tid == 0) atomicAdd(&a.sc->tc_timeouts, 1);
          st = ST_TIMEOUT;
          stop = true;
          break;
        }
        __syncthreads();
        if (tid == 0) hessian_timed(a.sc, th0);
        for (int r = tid; r < NM; r += NT) Hf[rowoff(NM) + r] = (float)s_g[r];
        __syncthreads();
        if (cholesky_aug<float>(Hf, NM, Pf, dinvf, &s_flag)) {
          float* xf = Pf;                                   // the panel buffers are free again
          for (int r = tid; r < NM; r += NT) xf[r] = -Hf[rowoff(NM) + r];
          __syncthreads();
          back_substitute<float>(Hf, NM, dinvf, xf);
          for (int r = tid; r < NM; r += NT) s_d[r] = (double)xf[r];
          __syncthreads();
          ++nfact;
          solved = true;
          have_factor = false;                              // the FP64 factor (if any) was overwritten
        } else if (tid == 0) {
          atomicAdd(&a.sc->fp32_fallbacks, 1);
        }
        __syncthreads();
      }
      if (solved) {
      } else if (reuse) {
        // chord step with the kept factor: L L^T Delta = -g
        for (int r = tid; r < NM; r += NT) s_d[r] = -s_g[r];
        __syncthreads();
        forward_substitute(s_H, NM, s_dinv, s_d);
        back_substitute(s_H, NM, s_dinv, s_d);
      } else {
      // (b) Hessian, packed lower triangle, row index r = i*M + a
      if (MIXED) {
        const uint64_t th0 = tid == 0 ? tc::globaltimer() : 0;
        if (!hessian_tc<M, double, SPLIT ? 2 : 1>(a, N, Qc, reinterpret_cast<const float*>(s_wJ), s_H, sA, sB, s_ph, tcs, &s_abort)) {
          if (tid == 0) atomicAdd(&a.sc->tc_timeouts, 1);
          st = ST_TIMEOUT;
          stop = true;
          break;
        }
        if (tid == 0) hessian_timed(a.sc, th0);
      } else {
        hessian_fp64<M>(a, N, Qc, s_wJ, s_H);
      }
      __syncthreads();
      if (a.h_dump) {
        const size_t NPH = (size_t)NM * (NM + 1) / 2;
        double* hd = a.h_dump + (size_t)wk * NPH;
        for (size_t r = tid; r < NPH; r += NT) hd[r] = s_H[r];
        break;
      }

      // (c) Cholesky with the gradient as augmented row NM, then L^T Delta = -L^-1 g
      for (int r = tid; r < NM; r += NT) s_H[rowoff(NM) + r] = s_g[r];
      __syncthreads();
      if constexpr (SPLIT) {
        if (!cholesky_split(s_H, NM, s_P, s_dinv, &s_flag, ssp, tcs, &s_abort)) {
          if (s_abort) {
            if (tid == 0) atomicAdd(&a.sc->tc_timeouts, 1);
            st = ST_TIMEOUT;
            stop = true;
          } else {
            st = ST_NOTSPD;
          }
          break;
        }
      } else {
        if (!cholesky_aug(s_H, NM, s_P, s_dinv, &s_flag)) { st = ST_NOTSPD; break; }
      }
      have_factor = true;
      ++nfact;
      if (a.f_dump) {
        const size_t NPH = (size_t)NM * (NM + 1) / 2;
        double* fd = a.f_dump + (size_t)wk * NPH;
        for (size_t r = tid; r < NPH; r += NT) fd[r] = s_H[r];
        break;
      }
      for (int r = tid; r < NM; r += NT) s_d[r] = -s_H[rowoff(NM) + r];
      __syncthreads();
      back_substitute(s_H, NM, s_dinv, s_d);
      }
      // direction at the nodes, slope, Delta . u_hat
      for (int q = tid; q < Qc; q += NT) {
        double acc[M];
#pragma unroll
        for (int c = 0; c < M; ++c) acc[c] = 0.0;
#pragma unroll 4
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
        for (int q = tid; q < Qc; q += NT) {
          double L[M], ss;
#pragma unroll
          for (int c = 0; c < M; ++c) L[c] = fma(alpha, s_dLam[c * Q + q], s_Lam[c * Q + q]);
          const bool ok = Closure<ENT, M>::feasible_sstar(L, a.ent, ss);
          rr[0] = fma(wc[q], ss, rr[0]);
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
      alpha_prev = alpha;
      for (int r = tid; r < NM; r += NT) s_lam[r] = fma(alpha, s_d[r], s_lam[r]);
      __syncthreads();
      ++it;
    }

    // results: duals, nodal states at the final duals, counters, signal speed
    for (int r = tid; r < NM; r += NT) lam_g[r] = s_lam[r];
    double* un = a.unode + (size_t)cell * M * Q;
    if (a.q_eval) {
      // per-level rules: the states at the nodes the stencil's updates read beyond this cell's own rule
      // (the ansatz of the final duals evaluated there), zero beyond them
      const int qe = a.q_eval[cell];
      for (int q = Qc + tid; q < qe; q += NT) {
        double L[M], u[M], ss;
#pragma unroll
        for (int c = 0; c < M; ++c) L[c] = 0.0;
        for (int i = 0; i < N; ++i) {
          const double ph = PhiT[(size_t)i * Q + q];
#pragma unroll
          for (int c = 0; c < M; ++c) L[c] = fma(ph, s_lam[i * M + c], L[c]);
        }
        Closure<ENT, M>::template eval<false>(L, a.ent, u, nullptr, ss);
#pragma unroll
        for (int c = 0; c < M; ++c) s_u[c * Q + q] = u[c];
      }
      __syncthreads();
      for (int r = tid; r < M * Q; r += NT) un[r] = (r % Q) < qe ? s_u[r] : 0.0;
    } else {
      for (int r = tid; r < M * Q; r += NT) un[r] = s_u[r];
    }
    if (tid == 0) {
      a.iters[cell] = it;
      a.status[cell] = st;
      if (nfact) atomicAdd(&a.sc->factorizations, (unsigned long long)nfact);
    }
    if (a.hessian_reuse == 2 && nfact > 0 && st == ST_OK) {
      // keep the newest factor for the next solve of this cell
      double* fs = a.factor_store + (size_t)cell * a.factor_stride;
      const size_t nph = (size_t)NM * (NM + 1) / 2;
      for (size_t r = tid; r < nph; r += NT) fs[r] = s_H[r];
      for (int r = tid; r < NM; r += NT) fs[nph + r] = s_dinv[r];
      if (tid == 0) a.factor_valid[cell] = 1;
    }
    const bool keep_img = img_wr && st == ST_OK;
    if (keep_img)
      for (int r = tid; r < NM; r += NT) a.img_lam[(size_t)cell * NMX + r] = s_lam[r];
    if (a.track_speed || keep_img) {
      // wave speeds at the nodes of the rule this cell's update integrates with
      const int qs = (a.lev_w && a.level_next) ? a.lev_q[a.level_next[cell]] : Q;
      double smax = 0.0;
      for (int q = tid; q < qs; q += NT) {
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
        if (a.track_speed) atomic_max_pos(&a.sc->smax_bits, v);
        if (keep_img) {
          a.img_smax[cell] = v;
          a.img_valid[cell] = lev_c + 1;
        }
      }
    }
    if constexpr (PHYS != PHYS_EULER2D)
      if (a.lf_a) lf_fold<PHYS, M>(a, cell, s_Lam, s_dLam, s_P, s_lf_ready);
    __syncthreads();
  }

  if (TC) {
    // drain whatever is still outstanding (only after a timeout), then free tensor memory. If a drain
    // wait runs out too, an MMA or bulk copy may still write to this CTA's tensor or shared memory:
    // the tensor memory is then left allocated and the context is marked unusable (sticky flag read
    // by the host, which launches nothing more into it).
    bool drained = true;
    for (int k = 0; k < TC_BARS; ++k)
      if (tcs.pend[k]) drained = tc_wait(tcs, k) && drained;
    tc::fence_before_sync();
    drained = __syncthreads_and(drained);
    tc::fence_after_sync();
    if (!drained) {
      if (tid == 0) atomicExch(&a.sc->tc_stuck, 1);
    } else if (warp == 0) {
      tc::tmem_dealloc(tcs.tmem, (uint32_t)a.mx.tmem_cols);
    }
  }
}

// prepare = 1: raise the kernel's dynamic shared-memory limit (outside any stream capture);
// prepare = 0: launch.
template <int ENT, int PHYS, int M, bool MIXED, bool F32F, bool SPLIT>
static cudaError_t launch_t(const NewtonArgs* a, int grid, size_t smem, bool h_in_smem, cudaStream_t s, int prepare,
                            int* blocks_per_sm) {
  auto k = h_in_smem ? k_newton<ENT, PHYS, M, true, MIXED, F32F, SPLIT> : k_newton<ENT, PHYS, M, false, MIXED, F32F, SPLIT>;
  if (prepare) {
    cudaError_t e = raise_smem_limit(k, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, NT, smem);
  }
  k<<<grid, NT, smem, s>>>(*a);
  return cudaGetLastError();
}

template <typename F>
static cudaError_t dispatch(int ent, int phys, int m, F&& f) {
  using std::integral_constant;
  if (phys == PHYS_BURGERS && m == 1) {
    if (ent == ENT_BARRIER) return f(integral_constant<int, ENT_BARRIER>(), integral_constant<int, PHYS_BURGERS>(), integral_constant<int, 1>());
    if (ent == ENT_QUADRATIC) return f(integral_constant<int, ENT_QUADRATIC>(), integral_constant<int, PHYS_BURGERS>(), integral_constant<int, 1>());
  }
  if (phys == PHYS_EULER1D && m == 3) {
    if (ent == ENT_EULER) return f(integral_constant<int, ENT_EULER>(), integral_constant<int, PHYS_EULER1D>(), integral_constant<int, 3>());
    if (ent == ENT_QUADRATIC) return f(integral_constant<int, ENT_QUADRATIC>(), integral_constant<int, PHYS_EULER1D>(), integral_constant<int, 3>());
  }
  if (phys == PHYS_EULER2D && m == 4) {
    if (ent == ENT_EULER) return f(integral_constant<int, ENT_EULER>(), integral_constant<int, PHYS_EULER2D>(), integral_constant<int, 4>());
    if (ent == ENT_QUADRATIC) return f(integral_constant<int, ENT_QUADRATIC>(), integral_constant<int, PHYS_EULER2D>(), integral_constant<int, 4>());
  }
  return cudaErrorInvalidValue;
}

// Modes: 0 FP64; 1 mixed (tensor-core Hessian, FP64 blocked factorisation); 2 mixed with an FP32
// factorisation; 3 mixed with the split factorisation (tensor-core trailing updates); 4 FP64 Hessian with
// the split factorisation. prepare = 1: raise the shared-memory limit and report blocks per SM; 0: launch.
template <int MODE>
cudaError_t newton_mode_call(int ent, int phys, int m, const NewtonArgs* a, int grid, size_t smem, bool h_in_smem,
                             cudaStream_t s, int prepare, int* blocks_per_sm) {
  constexpr bool MIXED = MODE == 1 || MODE == 2 || MODE == 3;
  constexpr bool F32F = MODE == 2;
  constexpr bool SPLIT = MODE == 3 || MODE == 4;
  return dispatch(ent, phys, m, [&](auto E, auto P, auto MM) {
    constexpr int e_ = decltype(E)::value, p_ = decltype(P)::value, m_ = decltype(MM)::value;
    return launch_t<e_, p_, m_, MIXED, F32F, SPLIT>(a, grid, smem, h_in_smem, s, prepare, blocks_per_sm);
  });
}

extern template cudaError_t newton_mode_call<0>(int, int, int, const NewtonArgs*, int, size_t, bool, cudaStream_t, int, int*);
extern template cudaError_t newton_mode_call<1>(int, int, int, const NewtonArgs*, int, size_t, bool, cudaStream_t, int, int*);
extern template cudaError_t newton_mode_call<2>(int, int, int, const NewtonArgs*, int, size_t, bool, cudaStream_t, int, int*);
extern template cudaError_t newton_mode_call<3>(int, int, int, const NewtonArgs*, int, size_t, bool, cudaStream_t, int, int*);
extern template cudaError_t newton_mode_call<4>(int, int, int, const NewtonArgs*, int, size_t, bool, cudaStream_t, int, int*);

}  // namespace ipm
