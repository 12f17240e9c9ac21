// ipm_host.h -- host-side internals shared by the translation units of libipm.
#pragma once
#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/ipm.h"
#include "ipm_device.cuh"

namespace ipm {

// NVTX range over a host call (seen by profilers as a named region; nothing without a tool attached)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct HostTables {
  int p = 0, M = 0, N = 0, Q = 0;
  std::vector<int> indices;     // [N][p]
  std::vector<double> nodes;    // [Q][p]
  std::vector<double> w;        // [Q]
  std::vector<double> Phi;      // [Q][N]
  std::vector<double> PhiT;     // [N][Q]
  std::vector<uint32_t> pairs;  // [N(N+1)/2]
};

// 2-D mesh tables built on the host (update2d.cu): areas [ny][nx], x-faces [ny][nx+1] and
// y-faces [ny+1][nx] as (n_x, n_y, length), h = min area / longest face.
struct Mesh2DHost {
  std::vector<double> area, xf, yf;
  double h_min = 0.0;
};

void set_global_error(const std::string& msg);
const char* check_problem(const ipm_problem* problem, const ipm_basis* basis, const ipm_quadrature* quad);
void build_mesh2d(const ipm_problem& pr, Mesh2DHost& m);
void gauss_legendre_1d(int n, std::vector<double>& x, std::vector<double>& w);
void build_tables(int p, int M, int nq, HostTables& t);
void clenshaw_curtis_1d(int k, std::vector<double>& x, std::vector<double>& w);
// nested tensor Clenshaw-Curtis tables of level kmax; level_w[k]: the level-k weights of the first nodes
void build_tables_cc(int p, int M, int kmax, HostTables& t, std::vector<std::vector<double>>& level_w);
// Clenshaw-Curtis level of every refinement level (n of them, total degrees M0, M0+1, ...) from a
// quadrature description; nullptr when valid, else what is wrong
const char* cc_levels(const ipm_quadrature* quad, int M0, int n, int* out);

// Tiling of the mixed-precision Hessian (see MixedTiles) and its shared-memory needs.
struct MixedLayout {
  bool ok = false;          // the problem fits the tensor-core path
  int n_pad = 0, kc = 0, chunks = 0, tiles = 0, tpp = 0, tmem_cols = 0;
  int abuf = 1;             // A staging buffers (2: build of the next K-chunk overlaps the MMAs)
  bool stack = false;       // B = [B_hi; B_lo] in one MMA operand (two accumulators of n_pad columns per row tile)
  size_t a_bytes = 0;       // A staging of one pass: abuf K-chunks (both BF16 terms each)
  size_t b_chunk_bytes = 0; // one K-chunk of the Phi image (both BF16 terms)
};
// Dynamic shared memory of the Newton kernel: byte offsets of the packed H, the A staging and
// the two Phi-chunk buffers, and the total.
struct NewtonSmem {
  uint32_t off_h = 0, off_a = 0, off_b = 0;
  uint32_t off_s = 0;       // digit slices and row exponents of the split factorisation
  size_t bytes = 0;
};

// Largest dynamic shared memory a kernel of this library may be launched with on the current
// device (the opt-in maximum). cudaFuncAttributeMaxDynamicSharedMemorySize is a property of the
// kernel function shared by every context and thread, so it is only ever set to this one value:
// a context with a smaller need can never lower the limit under another context's launches.
int max_dynamic_smem();

// Raise kernel k's dynamic shared-memory limit to the most it can have next to its static shared
// memory (the same value from every caller); fails with cudaErrorInvalidValue if `need` bytes do not fit.
template <typename K>
cudaError_t raise_smem_limit(K k, size_t need) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, k);
  if (e != cudaSuccess) return e;
  const int limit = max_dynamic_smem() - (int)fa.sharedSizeBytes;
  if ((long long)need > (long long)limit) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, limit);
}

// kernel launchers (newton.cu, update.cu)
// s_rows > 0: room for the split factorisation's digit slices (rows per slice from split_rows)
NewtonSmem newton_smem(int N, int m, int Q, bool h_in_smem, const MixedLayout* mx, int s_rows = 0);
MixedLayout mixed_layout(int N, int m, int Q, size_t smem_budget, bool h_in_smem, int s_rows = 0);
// rows per digit slice of the split factorisation of an N*m system, and the bytes of the slices
int split_rows(int NM);
size_t split_bytes(int rows);
constexpr int SPLIT_AUTO_NM = 128;         // factorization = 0: the split factorisation from this N*m (mixed)
constexpr int SPLIT_TMEM_COLS_ONE = 256;   // tensor-memory columns of one accumulator set
int newton_threads();
// mode: 0 FP64, 1 mixed (tensor-core Hessian, FP64 factorisation), 2 mixed with an FP32 factorisation,
// 3 mixed with the split factorisation (tensor-core trailing updates), 4 FP64 Hessian with the split one
cudaError_t launch_newton_phys(int ent, int phys, int m, const NewtonArgs& a, int grid, size_t smem, bool h_in_smem,
                               int mode, cudaStream_t s);
cudaError_t prepare_newton(int ent, int phys, int m, size_t smem, bool h_in_smem, int mode, int* blocks_per_sm);
// warp-per-cell Newton kernel for small cells (newton_warp.cu)
size_t newton_warp_slice(int N, int m, int Q);
cudaError_t prepare_newton_warp(int ent, int phys, int m, bool mixed, int warps, int slice, int* blocks_per_sm);
cudaError_t launch_newton_warp(int ent, int phys, int m, bool mixed, const NewtonArgs& a, int grid, int warps, int slice,
                               cudaStream_t s);
// level != nullptr: the cells of the levels below warp_levels are ordered after all others and
// sc->n_cta_items counts the others
cudaError_t launch_order(const int* iters, int n_work, int nx, int gy, int* order, cudaStream_t s,
                         const int* level = nullptr, int warp_levels = 0, StepScalars* sc = nullptr);
// one warp per cell with the nodes in chunks, for the small cells of adaptive meshes (newton_warpq.cu)
size_t newton_warpq_slice(int nm, int m);
cudaError_t prepare_newton_warpq(int ent, int phys, int m, bool mixed, int warps, int slice, int* blocks_per_sm);
cudaError_t launch_newton_warpq(int ent, int phys, int m, bool mixed, const NewtonArgs& a, int grid, int warps,
                                int slice, int nm_slice, cudaStream_t s);
cudaError_t launch_phi_images(const double* PhiT, int N, int Q, const MixedLayout& L, float* phiT32, float* phi32c,
                              uint8_t* img, cudaStream_t s);
cudaError_t prepare_update1d(int phys, int m, int N, int Q);
cudaError_t launch_update1d(int phys, int m, const Update1DArgs& a, int grid, cudaStream_t s);
// u_hat_j = lf_a[j] - (dt/dx) lf_b[j] on the interior cells (the Lax-Friedrichs update folded into the
// Newton launch), with the ghost copies and residual of launch_update1d
cudaError_t launch_lf_combine(const Update1DArgs& a, int NM, const double* lf_a, const double* lf_b, int grid,
                              cudaStream_t s);
cudaError_t launch_init1d(int ent, int m, const Tables& tab, const EntParams& ent_p, const ipm_problem& prob,
                          double* uhat, double* lam, int n_cells, cudaStream_t s);
cudaError_t launch_finalize(StepScalars* sc, const int* iters, const int* status, const double* cell_resid,
                            int n_cells, int first, int count, int advance_time, cudaStream_t s);
cudaError_t prepare_update2d(int N, int Q);
cudaError_t launch_update2d(const Update2DArgs& a, int grid, cudaStream_t s);
cudaError_t launch_init_levels(const Update2DArgs& a, int n_cells, cudaStream_t s);
cudaError_t launch_cap_levels(const Update2DArgs& a, int cap, cudaStream_t s);
// level != nullptr: project every cell at its level (lev_n moments) with its level's rule (lev_q nodes,
// weights lev_w [level][tab.Q])
cudaError_t launch_init2d(int ent, const Tables& tab, const EntParams& ent_p, const ipm_problem& prob, double* uhat,
                          double* lam, cudaStream_t s, const int* level = nullptr, const int* lev_n = nullptr,
                          const int* lev_q = nullptr, const double* lev_w = nullptr);
// adaptive meshes: the new level of every interior cell (Eq. errorIndicator on u_hat^n, capped), and with
// per-level rules the nodes each cell's nodal states must cover
cudaError_t launch_next_levels(const Update2DArgs& a, cudaStream_t s);
cudaError_t launch_bc_copy1d(double* uhat, double* lam, int nx, int Nm, int bc_left, int bc_right,
                             cudaStream_t s);

}  // namespace ipm
