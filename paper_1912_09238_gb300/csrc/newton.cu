// newton.cu -- host side of the per-cell Newton solve (the kernel template is in newton_kernel.cuh,
// instantiated per mode in newton_m*.cu): shared-memory and tensor-core layouts, launch dispatch by
// mode, the longest-first queue order (k_order) and the Phi images of the mixed path (k_phi_images).
#include "newton_kernel.cuh"

namespace ipm {

int newton_threads() { return NT; }

int max_dynamic_smem() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
  return v;
}

static size_t align128(size_t x) { return (x + 127) & ~size_t(127); }

int split_rows(int NM) {
  const int r = std::max(NM + 1 - SNB, 128);
  return (r + SBLK - 1) / SBLK * SBLK;
}

size_t split_bytes(int rows) { return align128((size_t)SDIG * rows * 32 + (size_t)rows * sizeof(int)); }

NewtonSmem newton_smem(int N, int m, int Q, bool h_in_smem, const MixedLayout* mx, int s_rows) {
  NewtonSmem s;
  const size_t NM = (size_t)N * m;
  const size_t B = (size_t)m * (m + 1) / 2;
  const size_t wj = mx ? (B * Q + 1) / 2 : B * Q;     // w J: float on the mixed path
  const size_t fixed =
      (4 * NM + 4 * (size_t)m * Q + wj + NWARPS * 8 + NM + 2 * (NM + 1) * PSTR) * sizeof(double);
  const size_t h_bytes = h_in_smem ? packed_aug_count((int)NM) * sizeof(double) : 0;
  s.off_h = (uint32_t)align128(fixed);
  const size_t sp_bytes = s_rows > 0 ? split_bytes(s_rows) : 0;
  if (!mx) {
    s.bytes = s.off_h + h_bytes;
    if (sp_bytes) {
      s.off_s = (uint32_t)align128(s.bytes);
      s.bytes = s.off_s + sp_bytes;
    }
    return s;
  }
  // With one pass the A staging may alias the packed H: H is written only after the last MMA of
  // the pass has completed. With several passes a later pass would overwrite the H entries of an
  // earlier one, so the staging gets its own region.
  const bool alias = h_in_smem && mx->tpp >= mx->tiles;
  const size_t region = alias ? std::max(h_bytes, mx->a_bytes) : h_bytes;
  s.off_a = alias ? s.off_h : (uint32_t)align128(s.off_h + h_bytes);
  s.off_b = (uint32_t)align128(alias ? s.off_h + region : s.off_a + mx->a_bytes);
  s.bytes = s.off_b + 2 * mx->b_chunk_bytes;
  if (sp_bytes) {
    // the digit slices of the split factorisation are live only during the factorisation, after the
    // Hessian's last MMA: they reuse the A staging when it has a region of its own and is large enough
    if (!alias && mx->a_bytes >= sp_bytes) {
      s.off_s = s.off_a;
    } else {
      s.off_s = (uint32_t)align128(s.bytes);
      s.bytes = s.off_s + sp_bytes;
    }
  }
  return s;
}

MixedLayout mixed_layout(int N, int m, int Q, size_t smem_budget, bool h_in_smem, int s_rows) {
  MixedLayout L;
  const int B = m * (m + 1) / 2;
  L.n_pad = (N + 15) / 16 * 16;
  L.kc = Q > 16 ? 32 : 16;
  L.chunks = (Q + L.kc - 1) / L.kc;
  L.tiles = (B * N + 127) / 128;
  L.b_chunk_bytes = (size_t)2 * L.n_pad * L.kc * 2;
  if (L.n_pad > 256) return L;
  // B = [B_hi; B_lo] as one operand of 2 n_pad rows (two accumulators per row tile) when that needs no
  // more passes over the row tiles than one accumulator per tile does
  {
    auto passes = [&](int cols) { return (L.tiles + std::min(L.tiles, 512 / cols) - 1) / std::min(L.tiles, 512 / cols); };
    L.stack = 2 * L.n_pad <= 256 && passes(2 * L.n_pad) == passes(L.n_pad);
  }
  const int acc_cols = L.stack ? 2 * L.n_pad : L.n_pad;
  // row tiles per pass: bounded by tensor memory (512 columns) and by the shared-memory budget
  // (two A buffers when they fit at that tile count, else one)
  for (int tpp = std::min(L.tiles, 512 / acc_cols); tpp >= 1; --tpp) {
   for (int abuf = L.chunks > 1 ? 2 : 1; abuf >= 1; --abuf) {
    L.tpp = tpp;
    L.abuf = abuf;
    L.a_bytes = (size_t)abuf * 2 * tpp * 128 * L.kc * 2;
    if (newton_smem(N, m, Q, h_in_smem, &L, s_rows).bytes <= smem_budget) {
      int cols = 32;
      while (cols < tpp * acc_cols) cols *= 2;
      if (s_rows > 0) cols = std::max(cols, SPLIT_BUF_COLS);   // one accumulator set of the split factorisation
      L.tmem_cols = cols;
      L.ok = true;
      return L;
    }
   }
  }
  L.tpp = 0;
  return L;
}

static cudaError_t newton_call(int mode, int ent, int phys, int m, const NewtonArgs* a, int grid, size_t smem,
                               bool h_in_smem, cudaStream_t s, int prepare, int* blocks_per_sm) {
  switch (mode) {
    case 0: return newton_mode_call<0>(ent, phys, m, a, grid, smem, h_in_smem, s, prepare, blocks_per_sm);
    case 1: return newton_mode_call<1>(ent, phys, m, a, grid, smem, h_in_smem, s, prepare, blocks_per_sm);
    case 2: return newton_mode_call<2>(ent, phys, m, a, grid, smem, h_in_smem, s, prepare, blocks_per_sm);
    case 3: return newton_mode_call<3>(ent, phys, m, a, grid, smem, h_in_smem, s, prepare, blocks_per_sm);
    case 4: return newton_mode_call<4>(ent, phys, m, a, grid, smem, h_in_smem, s, prepare, blocks_per_sm);
    default: return cudaErrorInvalidValue;
  }
}

// mode: see newton_mode_call
cudaError_t prepare_newton(int ent, int phys, int m, size_t smem, bool h_in_smem, int mode, int* blocks_per_sm) {
  return newton_call(mode, ent, phys, m, nullptr, 0, smem, h_in_smem, nullptr, 1, blocks_per_sm);
}

cudaError_t launch_newton_phys(int ent, int phys, int m, const NewtonArgs& a, int grid, size_t smem, bool h_in_smem,
                               int mode, cudaStream_t s) {
  return newton_call(mode, ent, phys, m, &a, grid, smem, h_in_smem, s, 0, nullptr);
}

// Longest-first order of the Newton work queue: the work items (interior cells, mapped as in the
// Newton kernel) sorted by the largest Newton count of the cell and its face neighbours in the previous
// solve, descending; ties in any order.
// The order decides only which CTA takes which cell when: each cell's arithmetic is independent of
// it, so results do not depend on it. One CTA; warp-aggregated shared-memory atomics.
constexpr int ORDER_KEYS = 256;   // two groups of 128 predicted counts
constexpr int ORDER_T = 1024;

__global__ void __launch_bounds__(ORDER_T) k_order(const int* __restrict__ iters, int n_work, int nx, int gy,
                                                   int* __restrict__ order, const int* __restrict__ level,
                                                   int warp_levels, StepScalars* sc) {
  __shared__ int cnt[ORDER_KEYS];
  const int tid = threadIdx.x, lane = tid & 31;
  for (int k = tid; k < ORDER_KEYS; k += ORDER_T) cnt[k] = 0;
  __syncthreads();
  for (int pass = 0; pass < 2; ++pass) {
    for (int base = 0; base < n_work; base += ORDER_T) {
      const int w = base + tid;
      const bool valid = w < n_work;
      const int cell = valid ? work_cell(w, nx, gy) : 0;
      // predicted work: the most Newton updates the cell or a face neighbour needed in the last solve (a
      // discontinuity moves less than a cell per step, so the cells it is about to enter start early too)
      int pred = 0;
      if (valid) {
        pred = max(iters[cell], max(iters[cell - 1], iters[cell + 1]));
        if (gy) pred = max(pred, max(iters[cell - (nx + 2)], iters[cell + (nx + 2)]));
      }
      // split queue (adaptive meshes): the cells of the levels below warp_levels form the second group
      const int group = (valid && level && level[cell] < warp_levels) ? 1 : 0;
      const int key = valid ? group * 128 + 127 - min(max(pred, 0), 127) : -1;
      const unsigned peers = __match_any_sync(0xffffffffu, key);
      const int leader = __ffs(peers) - 1;
      const int rank = __popc(peers & ((1u << lane) - 1u));
      int at = 0;
      if (valid && lane == leader) at = atomicAdd(&cnt[key], __popc(peers));
      at = __shfl_sync(0xffffffffu, at, leader);
      if (pass == 1 && valid) order[at + rank] = cell;
    }
    __syncthreads();
    if (pass == 0 && tid == 0) {
      // counts -> starting offsets (key 0 = most iterations first)
      int run = 0;
      for (int k = 0; k < ORDER_KEYS; ++k) {
        const int c = cnt[k];
        cnt[k] = run;
        run += c;
      }
      if (sc) sc->n_cta_items = cnt[128];   // the first group ends where the second begins
    }
    __syncthreads();
  }
}

cudaError_t launch_order(const int* iters, int n_work, int nx, int gy, int* order, cudaStream_t s, const int* level,
                         int warp_levels, StepScalars* sc) {
  k_order<<<1, ORDER_T, 0, s>>>(iters, n_work, nx, gy, order, level, warp_levels, sc);
  return cudaGetLastError();
}

// Phi in the forms the mixed path reads: FP32 Phi^T [N][Q], the same by K-chunk with rows padded to
// kc + 4 floats ([chunk][N][kc + 4], zero beyond Q), and per K-chunk the two BF16 terms (hi, lo) of
// B[j][k] = phi_j(xi_k) in the K-major tile layout (zero beyond N and Q).
__global__ void k_phi_images(const double* __restrict__ PhiT, int N, int Q, int n_pad, int kc, int chunks,
                             float* __restrict__ phiT32, float* __restrict__ phi32c, uint8_t* __restrict__ img) {
  const uint32_t sbo = tc::kmajor_sbo(kc);
  const size_t b_img = (size_t)n_pad * kc * 2;
  const int total = chunks * n_pad * kc;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int c = idx / (n_pad * kc);
    const int rem = idx - c * n_pad * kc;
    const int j = rem / kc, k = rem - j * kc;
    const int q = c * kc + k;
    const float x = (j < N && q < Q) ? (float)PhiT[(size_t)j * Q + q] : 0.f;
    if (j < N && q < Q) phiT32[(size_t)j * Q + q] = x;
    if (j < N) {
      float* row = phi32c + ((size_t)c * N + j) * (kc + 4);
      row[k] = x;
      if (k < 4) row[kc + k] = 0.f;
    }
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    uint8_t* base = img + (size_t)c * 2 * b_img;
    const uint32_t off = tc::kmajor_offset(j, k, sbo);
    *reinterpret_cast<__nv_bfloat16*>(base + off) = h;
    *reinterpret_cast<__nv_bfloat16*>(base + b_img + off) = l;
  }
}

cudaError_t launch_phi_images(const double* PhiT, int N, int Q, const MixedLayout& L, float* phiT32, float* phi32c,
                              uint8_t* img, cudaStream_t s) {
  const int total = L.chunks * L.n_pad * L.kc;
  k_phi_images<<<std::max(1, std::min(1024, (total + 255) / 256)), 256, 0, s>>>(PhiT, N, Q, L.n_pad, L.kc, L.chunks,
                                                                                 phiT32, phi32c, img);
  return cudaGetLastError();
}

}  // namespace ipm
