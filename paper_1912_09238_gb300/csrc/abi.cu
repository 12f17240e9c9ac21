// abi.cu -- the extern "C" entry points of libipm (declared and documented in include/ipm.h).
//
// A context owns the resident device state of one IPM problem: tables (Phi, Phi^T, weights,
// nodes, moment pairs), moments u_hat and duals lambda [cell][moment][variable], nodal states
// [cell][variable][node], per-cell counters, the step scalars, and the CUDA graphs of one
// Algorithm-1 step and one Algorithm-2 step.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "ipm_host.h"

using namespace ipm;

struct ipm_ctx {
  ipm_problem prob;
  ipm_basis basis;
  ipm_quadrature quad;
  ipm_entropy ent;
  ipm_options opt;
  HostTables tab;
  int m = 0, N = 0, Q = 0, NM = 0, n_cells = 0, n_interior = 0;
  int phys = 0, entk = 0;
  double dx = 0.0;
  bool is2d = false;
  Mesh2DHost mesh2d;
  int n_levels = 0;                 // adaptive: levels adapt_min_degree .. total_degree
  int lev_n[8] = {0}, lev_prev[8] = {0};
  int* d_level = nullptr;
  int* d_level_next = nullptr;      // adaptive: the new level of every cell, set before each Newton launch
  // quadrature per level (IPM_QUAD_CC_NESTED on an adaptive mesh): nodes and weights [level][Q] of each
  // level's rule; without it every level uses the table's rule
  bool level_rules = false;
  int lev_q[8] = {0};
  std::vector<double> lev_w;
  double* d_lev_w = nullptr;
  int* d_q_eval = nullptr;          // nodes each cell's nodal states must cover (per-level rules)
  double* d_factors = nullptr;      // hessian_reuse 2: kept Cholesky factors per cell
  int* d_factor_valid = nullptr;
  size_t factor_stride = 0;
  // moment images per cell (fixed-degree meshes, check_cache != 0): the convergence check of a cell whose
  // duals did not move since its last solve comes from them (CTA-per-cell Newton kernel)
  bool img = false;
  double *d_img = nullptr, *d_img_lam = nullptr, *d_img_smax = nullptr;
  int* d_img_valid = nullptr;
  // 1-D meshes: the Lax-Friedrichs terms the CTA-per-cell Newton launch folds in (A, B per cell) and
  // the per-cell counts of finished neighbours
  double *d_lf_a = nullptr, *d_lf_b = nullptr;
  int* d_lf_cnt = nullptr;
  double *d_area = nullptr, *d_xf = nullptr, *d_yf = nullptr;
  int device = 0;
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;
  // device state
  double *d_Phi = nullptr, *d_PhiT = nullptr, *d_w = nullptr, *d_nodes = nullptr;
  uint32_t* d_pairs = nullptr;
  double *d_uhat = nullptr, *d_lam = nullptr, *d_unode = nullptr, *d_cell_resid = nullptr, *d_hwork = nullptr;
  int *d_iters = nullptr, *d_status = nullptr, *d_ghost_list = nullptr;
  int* d_order = nullptr;       // longest-first Newton queue of the interior cells
  StepScalars* d_sc = nullptr;
  int n_fixed_ghosts = 0;
  // launch configuration
  bool mixed = false;          // precision IPM_PREC_MIXED or _MIXED_F32_FACTOR: tensor-core Hessian
  int newton_mode = 0;         // 0 FP64, 1 mixed, 2 mixed with an FP32 factorisation, 3 mixed + split, 4 FP64 + split
  bool split = false;          // split factorisation (tensor-core trailing updates) on the CTA-per-cell kernel
  int s_rows = 0, s_nbuf = 0;  // its digit-slice rows and tensor-memory accumulator sets
  uint32_t ph_stage_off = 0;    // shared-memory offset of the staged Phi^T chunks of the mixed Hessian (0: none)
  MixedLayout mx;
  NewtonSmem sm;
  float* d_phiT32 = nullptr;
  float* d_phi32c = nullptr;     // [chunk][N][kc + 4] Phi^T by K-chunk (staged by bulk copy)
  uint8_t* d_phi_img = nullptr;
  size_t newton_smem = 0;
  bool h_in_smem = true;
  // Newton kernel variant: 0 = one CTA per cell (newton.cu), 1 = one warp per cell (newton_warp.cu,
  // N*m <= 64), picked at init by timing both on the initial state
  int newton_kind = 0;
  int warp_warps = 0, warp_slice = 0, warp_grid = 0;
  float tune_ms[3] = {0.f, 0.f, 0.f};
  int newton_grid = 0;
  // adaptive meshes: the cells of the lowest warp_levels levels (N m <= 64) are solved one warp per cell
  // (newton_warpq.cu) before the CTA-per-cell kernel takes the others
  int warp_levels = 0;
  int wq_warps = 0, wq_slice = 0, wq_nm = 0, wq_grid = 0;
  size_t hwork_stride = 0;
  int update_grid = 0;
  // timing events recorded inside every step (begin, after Newton, after update, end)
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  // graphs
  cudaGraphExec_t step_exec = nullptr;
  cudaGraphExec_t oneshot_exec = nullptr;
  // set once a Newton CTA reported tensor-core work it could not drain (StepScalars::tc_stuck): its
  // tensor memory stays allocated and nothing more is launched into this context
  bool unusable = false;
  std::string err;
};

static std::mutex g_err_mu;
static std::string g_init_err;

namespace ipm {
// message for ipm_last_error(NULL) from calls that have no context
void set_global_error(const std::string& msg) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  g_init_err = msg;
}
}  // namespace ipm

static ipm_status fail(ipm_ctx* c, ipm_status s, const std::string& msg) {
  if (c) {
    c->err = msg;
  } else {
    std::lock_guard<std::mutex> lk(g_err_mu);
    g_init_err = msg;
  }
  return s;
}

// A failed call returns its status; a non-sticky error (e.g. an allocation that did not fit) is also
// cleared from the runtime's last-error slot, so that later launches of any context do not report it.
#define IPM_CK(ctx, call)                                                                               \
  do {                                                                                                  \
    cudaError_t e_ = (call);                                                                            \
    if (e_ != cudaSuccess) {                                                                            \
      cudaGetLastError();                                                                               \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? IPM_ENOMEM : IPM_ECUDA,                        \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                                 \
    }                                                                                                   \
  } while (0)

static Tables dev_tables(const ipm_ctx* c) {
  Tables t;
  t.Phi = c->d_Phi;
  t.PhiT = c->d_PhiT;
  t.w = c->d_w;
  t.nodes = c->d_nodes;
  t.pairs = c->d_pairs;
  t.N = c->N;
  t.Q = c->Q;
  t.p = c->tab.p;
  return t;
}

static EntParams ent_params(const ipm_ctx* c) {
  EntParams e;
  e.u_minus = c->ent.u_minus;
  e.u_plus = c->ent.u_plus;
  e.gamma = c->prob.gamma;
  return e;
}

static NewtonArgs newton_args(const ipm_ctx* c, int one_step) {
  NewtonArgs a;
  a.tab = dev_tables(c);
  a.ent = ent_params(c);
  a.uhat = c->d_uhat;
  a.lam = c->d_lam;
  a.unode = c->d_unode;
  a.iters = c->d_iters;
  a.status = c->d_status;
  a.hwork = c->d_hwork;
  a.hwork_stride = c->hwork_stride;
  a.sc = c->d_sc;
  a.cell_list = nullptr;
  a.n_work = c->n_interior;
  a.nx = c->prob.nx;
  a.gy = c->is2d ? 1 : 0;
  a.one_step = one_step;
  a.tau = c->opt.newton_tol;
  a.armijo_c = c->opt.armijo_c;
  a.slack_rel = c->opt.slack_rel;
  a.max_newton = c->opt.max_newton;
  a.max_halvings = c->opt.max_halvings;
  a.track_speed = 1;
  a.h_dump = nullptr;
  a.hessian_reuse = c->opt.hessian_reuse;
  a.reuse_ratio = c->opt.reuse_ratio;
  a.factor_store = c->d_factors;
  a.factor_stride = c->factor_stride;
  a.factor_valid = c->d_factor_valid;
  a.level = c->n_levels ? c->d_level : nullptr;
  for (int k = 0; k < 8; ++k) {
    a.lev_n[k] = c->lev_n[k];
    a.lev_q[k] = c->lev_q[k];
  }
  a.lev_w = c->level_rules ? c->d_lev_w : nullptr;
  a.level_next = c->n_levels ? c->d_level_next : nullptr;
  a.q_eval = c->level_rules ? c->d_q_eval : nullptr;
  a.queue = nullptr;
  a.first_dev = nullptr;
  a.count_dev = nullptr;
  const bool img = c->img && c->newton_kind == 0;
  a.img = img ? c->d_img : nullptr;
  a.img_lam = img ? c->d_img_lam : nullptr;
  a.img_smax = img ? c->d_img_smax : nullptr;
  a.img_valid = img ? c->d_img_valid : nullptr;
  a.lf_a = nullptr;                // set by enqueue_step on 1-D meshes
  a.lf_b = nullptr;
  a.lf_cnt = nullptr;
  a.bc_left = c->prob.bc_left;
  a.bc_right = c->prob.bc_right;
  a.mx.phi_img = c->d_phi_img;
  a.mx.phiT32 = c->d_phiT32;
  a.mx.phi32c = c->d_phi32c;
  a.mx.n_rows = c->N;
  a.mx.kcp = c->mx.kc + 4;
  a.mx.off_ph = c->ph_stage_off;
  a.mx.n_pad = c->mx.n_pad;
  a.mx.kc = c->mx.kc;
  a.mx.chunks = c->mx.chunks;
  a.mx.tiles = c->mx.tiles;
  a.mx.tpp = c->mx.tpp;
  a.mx.tmem_cols = c->mx.tmem_cols;
  a.mx.abuf = c->mx.abuf;
  a.mx.stack = c->mx.stack ? 1 : 0;
  a.off_h = c->sm.off_h;
  a.off_a = c->sm.off_a;
  a.off_b = c->sm.off_b;
  a.off_s = c->sm.off_s;
  a.s_rows = c->s_rows;
  a.s_nbuf = c->s_nbuf;
  a.f_dump = nullptr;
  return a;
}

static Update1DArgs update_args(const ipm_ctx* c, double dt_override, bool resid) {
  Update1DArgs u;
  u.tab = dev_tables(c);
  u.uhat = c->d_uhat;
  u.lam = c->d_lam;
  u.unode = c->d_unode;
  u.cell_resid = resid ? c->d_cell_resid : nullptr;
  u.sc = c->d_sc;
  u.nx = c->prob.nx;
  u.bc_left = c->prob.bc_left;
  u.bc_right = c->prob.bc_right;
  u.dx = c->dx;
  u.cfl = c->prob.cfl;
  u.t_end = c->prob.t_end;
  u.gamma = c->prob.gamma;
  u.dt_override = dt_override;
  return u;
}

static Update2DArgs update2d_args(const ipm_ctx* c, double dt_override, bool resid, bool clip) {
  Update2DArgs u;
  u.tab = dev_tables(c);
  u.mesh.area = c->d_area;
  u.mesh.xf = c->d_xf;
  u.mesh.yf = c->d_yf;
  u.mesh.nx = c->prob.nx;
  u.mesh.ny = c->prob.ny;
  u.mesh.h_min = c->mesh2d.h_min;
  u.uhat = c->d_uhat;
  u.unode = c->d_unode;
  u.cell_resid = resid ? c->d_cell_resid : nullptr;
  u.sc = c->d_sc;
  u.bc[0] = c->prob.bc_left;
  u.bc[1] = c->prob.bc_right;
  u.bc[2] = c->prob.bc_bottom;
  u.bc[3] = c->prob.bc_top;
  u.cfl = c->prob.cfl;
  u.t_end = c->prob.t_end;
  u.gamma = c->prob.gamma;
  u.dt_override = dt_override;
  u.clip = clip ? 1 : 0;
  u.level = c->n_levels ? c->d_level : nullptr;
  u.lam = c->d_lam;
  u.n_levels = c->n_levels;
  for (int k = 0; k < 8; ++k) {
    u.lev_n[k] = c->lev_n[k];
    u.lev_prev[k] = c->lev_prev[k];
  }
  u.delta_lo = std::min(c->opt.delta_lo, c->opt.delta_hi);
  u.delta_hi = std::max(c->opt.delta_lo, c->opt.delta_hi);
  u.level_next = c->n_levels ? c->d_level_next : nullptr;
  u.q_eval = c->level_rules ? c->d_q_eval : nullptr;
  for (int k = 0; k < 8; ++k) u.lev_q[k] = c->lev_q[k];
  u.lev_w = c->level_rules ? c->d_lev_w : nullptr;
  return u;
}

// the Newton kernel of the context's chosen variant
static cudaError_t launch_newton_ctx(const ipm_ctx* c, const NewtonArgs& a, int n_work, cudaStream_t s) {
  if (c->newton_kind == 1) {
    const int grid = std::max(1, std::min(c->warp_grid, (n_work + c->warp_warps - 1) / c->warp_warps));
    return launch_newton_warp(c->entk, c->phys, c->m, c->mixed, a, grid, c->warp_warps, c->warp_slice, s);
  }
  return launch_newton_phys(c->entk, c->phys, c->m, a, std::max(1, std::min(c->newton_grid, n_work)), c->newton_smem,
                            c->h_in_smem, c->newton_mode, s);
}

// enqueue: queue reset, Newton over the interior
static cudaError_t enqueue_newton(ipm_ctx* c, int one_step, cudaStream_t s, bool lf = false) {
  cudaError_t e = cudaSuccess;
  if (c->n_levels) {
    // the levels of this step's update (from the moments the dual problems are solved for): the Newton
    // kernel evaluates each cell at the nodes its stencil's updates read and takes the wave speed there
    e = launch_next_levels(update2d_args(c, 0.0, false, false), s);
    if (e != cudaSuccess) return e;
  }
  e = cudaMemsetAsync(&c->d_sc->work_counter, 0, sizeof(int), s);
  if (c->warp_levels > 0) {
    // split queue: the small-level cells, one warp per cell, then the others, one CTA per cell
    if (e == cudaSuccess) e = cudaMemsetAsync(&c->d_sc->warp_counter, 0, sizeof(int), s);
    if (e == cudaSuccess)
      e = launch_order(c->d_iters, c->n_interior, c->prob.nx, 1, c->d_order, s, c->d_level, c->warp_levels, c->d_sc);
    if (e != cudaSuccess) return e;
    NewtonArgs a = newton_args(c, one_step);
    a.cell_list = c->d_order;
    a.queue = &c->d_sc->warp_counter;
    a.first_dev = &c->d_sc->n_cta_items;
    e = launch_newton_warpq(c->entk, c->phys, c->m, c->mixed, a, c->wq_grid, c->wq_warps, c->wq_slice, c->wq_nm, s);
    if (e != cudaSuccess) return e;
    a.queue = nullptr;
    a.first_dev = nullptr;
    a.count_dev = &c->d_sc->n_cta_items;
    return launch_newton_ctx(c, a, c->n_interior, s);
  }
  if (e == cudaSuccess) e = launch_order(c->d_iters, c->n_interior, c->prob.nx, c->is2d ? 1 : 0, c->d_order, s);
  if (e == cudaSuccess && lf) e = cudaMemsetAsync(c->d_lf_cnt, 0, (size_t)c->n_cells * sizeof(int), s);
  if (e != cudaSuccess) return e;
  NewtonArgs a = newton_args(c, one_step);
  a.cell_list = c->d_order;
  if (lf) {
    a.lf_a = c->d_lf_a;
    a.lf_b = c->d_lf_b;
    a.lf_cnt = c->d_lf_cnt;
  }
  return launch_newton_ctx(c, a, c->n_interior, s);
}

// one step of Algorithm 1 (one_step = 0) or Algorithm 2 (one_step = 1)
static cudaError_t enqueue_step(ipm_ctx* c, int one_step, cudaStream_t s) {
  // 1-D meshes: the Newton launch folds in the Lax-Friedrichs terms and a small kernel applies dt
  const bool lf = !c->is2d && c->d_lf_a != nullptr;
  cudaError_t e = cudaEventRecordWithFlags(c->ev[0], s, cudaEventRecordExternal);
  if (e == cudaSuccess) e = enqueue_newton(c, one_step, s, lf);
  if (e == cudaSuccess) e = cudaEventRecordWithFlags(c->ev[1], s, cudaEventRecordExternal);
  if (e != cudaSuccess) return e;
  if (c->is2d) {
    e = launch_update2d(update2d_args(c, 0.0, true, one_step == 0), c->update_grid, s);
  } else if (lf) {
    e = launch_lf_combine(update_args(c, 0.0, true), c->NM, c->d_lf_a, c->d_lf_b, c->update_grid, s);
  } else {
    Update1DArgs u = update_args(c, 0.0, true);
    e = launch_update1d(c->phys, c->m, u, c->update_grid, s);
  }
  if (e == cudaSuccess) e = cudaEventRecordWithFlags(c->ev[2], s, cudaEventRecordExternal);
  // 2-D interior cells are not contiguous: reduce over every cell (ghost counters are kept at zero)
  const int first = c->is2d ? 0 : 1, count = c->is2d ? c->n_cells : c->n_interior;
  if (e == cudaSuccess) e = launch_finalize(c->d_sc, c->d_iters, c->d_status, c->d_cell_resid, c->n_cells, first, count, 1, s);
  if (e == cudaSuccess) e = cudaEventRecordWithFlags(c->ev[3], s, cudaEventRecordExternal);
  return e;
}

// Process-wide record of tuning decisions, keyed by everything that shapes the Newton launch: a
// problem of the same shape reuses the first decision, so its results do not depend on the load the
// GPU happened to carry when it was tuned (and serving does not re-tune every request).
struct TuneKey {
  int kind, entk, N, m, Q, mixed, size_bucket;
  bool operator<(const TuneKey& o) const {
    return std::tie(kind, entk, N, m, Q, mixed, size_bucket) < std::tie(o.kind, o.entk, o.N, o.m, o.Q, o.mixed, o.size_bucket);
  }
};
// Device memory of a context comes from one stream-ordered memory pool per device
// (cudaMallocFromPoolAsync / cudaFreeAsync on the context's stream). Creating or destroying a context
// therefore neither calls cudaMalloc nor cudaFree, whose implicit synchronisation would stall the work
// of every other context on the device (the serving layer creates and destroys contexts while others
// run). Freed blocks stay in the pool (no release threshold) and serve the next context.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64] = {};

static cudaError_t device_pool(int dev, cudaMemPool_t* out) {
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    cudaError_t e = cudaMemPoolCreate(&p, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = ~0ull;
    e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(p);
      return e;
    }
    g_pool[dev] = p;
  }
  *out = g_pool[dev];
  return cudaSuccess;
}

// Device memory a new context can still obtain: what the device reports free plus what the pool holds
// for reuse (blocks freed by earlier contexts count as used in the device's report).
static cudaError_t available_device_bytes(size_t* out) {
  int dev = 0;
  size_t free_b = 0, total_b = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
  if (e != cudaSuccess) return e;
  cudaMemPool_t pool = nullptr;
  e = device_pool(dev, &pool);
  if (e != cudaSuccess) return e;
  uint64_t reserved = 0, used = 0;
  e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved);
  if (e == cudaSuccess) e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used);
  if (e != cudaSuccess) return e;
  *out = free_b + (size_t)(reserved > used ? reserved - used : 0);
  return cudaSuccess;
}

// bytes of device memory for the context, ordered on stream s (default: the context's own stream)
template <typename T>
static cudaError_t dalloc(const ipm_ctx* c, T** p, size_t bytes, cudaStream_t s = nullptr) {
  if (!s) s = c->own_stream;
  cudaMemPool_t pool = nullptr;
  cudaError_t e = device_pool(c->device, &pool);
  if (e != cudaSuccess) return e;
  return cudaMallocFromPoolAsync(reinterpret_cast<void**>(p), std::max<size_t>(bytes, 1), pool, s);
}

struct TuneVal {
  int kind;
  float ms[2];
};
static std::mutex g_tune_mu;
static std::map<TuneKey, TuneVal> g_tune;

// Time one Newton solve of the interior on the initial state with each applicable kernel variant
// (the duals are restored after every trial) and keep the fastest. Ties go to the CTA kernel.
static ipm_status autotune_newton(ipm_ctx* c) {
  // the interior size enters as its power-of-two bucket: meshes of similar size share a decision
  int size_bucket = 0;
  while ((1 << (size_bucket + 1)) <= c->n_interior) ++size_bucket;
  const TuneKey key{c->prob.kind, c->entk, c->N, c->m, c->Q, c->mixed ? 1 : 0, size_bucket};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      c->newton_kind = it->second.kind;
      c->tune_ms[0] = it->second.ms[0];
      c->tune_ms[1] = it->second.ms[1];
      return IPM_OK;
    }
  }
  const size_t bytes = (size_t)c->n_cells * c->NM * sizeof(double);
  double* saved = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  IPM_CK(c, dalloc(c, &saved, bytes, c->stream));
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaMemcpyAsync(saved, c->d_lam, bytes, cudaMemcpyDeviceToDevice, c->stream);
  float best = 1e30f;
  int best_kind = 0;
  for (int kind = 0; kind < 2 && e == cudaSuccess; ++kind) {
    c->newton_kind = kind;
    float ms = 0.f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // the first run warms the kernel up
      e = cudaMemcpyAsync(c->d_lam, saved, bytes, cudaMemcpyDeviceToDevice, c->stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(&c->d_sc->work_counter, 0, sizeof(int), c->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
      if (e == cudaSuccess) {
        NewtonArgs a = newton_args(c, 0);
        a.track_speed = 0;
        // both variants evaluate every check: the timing compares the kernels, not the image cache
        a.img = nullptr;
        a.img_lam = nullptr;
        a.img_smax = nullptr;
        a.img_valid = nullptr;
        e = launch_newton_ctx(c, a, c->n_interior, c->stream);
      }
      if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    c->tune_ms[kind] = ms;
    if (e == cudaSuccess && ms < best * 0.97f) {
      best = ms;
      best_kind = kind;
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_lam, saved, bytes, cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(&c->d_sc->work_counter, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_iters, 0, (size_t)c->n_cells * sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  c->newton_kind = best_kind;
  if (e == cudaSuccess) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.emplace(key, TuneVal{best_kind, {c->tune_ms[0], c->tune_ms[1]}});
  }
  cudaFreeAsync(saved, c->stream);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  IPM_CK(c, e);
  return IPM_OK;
}

static ipm_status build_graph(ipm_ctx* c, int one_step, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  IPM_CK(c, cudaStreamBeginCapture(c->own_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = enqueue_step(c, one_step, c->own_stream);
  cudaError_t e2 = cudaStreamEndCapture(c->own_stream, &g);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(c, IPM_ECUDA, std::string("capture of the step: ") + cudaGetErrorString(e));
  }
  IPM_CK(c, e2);
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  IPM_CK(c, e);
  return IPM_OK;
}

static void free_ctx(ipm_ctx* c) {
  if (!c) return;
  if (c->step_exec) cudaGraphExecDestroy(c->step_exec);
  for (cudaEvent_t ev : c->ev)
    if (ev) cudaEventDestroy(ev);
  if (c->oneshot_exec) cudaGraphExecDestroy(c->oneshot_exec);
  void* ptrs[] = {c->d_Phi, c->d_PhiT, c->d_w, c->d_nodes, c->d_pairs, c->d_uhat, c->d_lam, c->d_unode,
                  c->d_cell_resid, c->d_hwork, c->d_iters, c->d_status, c->d_ghost_list, c->d_sc,
                  c->d_phiT32, c->d_phi32c, c->d_phi_img, c->d_order, c->d_area, c->d_xf, c->d_yf, c->d_level,
                  c->d_factors, c->d_factor_valid, c->d_level_next, c->d_lev_w, c->d_q_eval,
                  c->d_img, c->d_img_lam, c->d_img_smax, c->d_img_valid, c->d_lf_a, c->d_lf_b, c->d_lf_cnt};
  cudaStream_t fs = c->stream ? c->stream : c->own_stream;
  for (void* p : ptrs)
    if (p) cudaFreeAsync(p, fs);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  delete c;
}

// a device copy of a host vector on the context's own stream (the pageable source is staged before the
// call returns)
template <typename T>
static cudaError_t upload(const ipm_ctx* c, T** dst, const std::vector<T>& src) {
  cudaError_t e = dalloc(c, dst, src.size() * sizeof(T), c->own_stream);
  if (e != cudaSuccess) return e;
  if (src.empty()) return cudaSuccess;
  return cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, c->own_stream);
}

namespace ipm {
// Checks of a problem, its basis and its quadrature shared by every entry point that takes them;
// nullptr when they are valid, else what is wrong.
const char* check_problem(const ipm_problem* problem, const ipm_basis* basis, const ipm_quadrature* quad) {
  if (basis->p < 1 || basis->p > 3 || basis->total_degree < 0)
    return "basis needs 1 <= p <= 3, M >= 0";
  if (quad->kind != IPM_QUAD_GAUSS && quad->kind != IPM_QUAD_CC_NESTED) return "unknown quadrature kind";
  if (quad->kind == IPM_QUAD_GAUSS && quad->n_per_dim < 1) return "a Gauss rule needs n_per_dim >= 1";
  if (problem->kind != IPM_BURGERS_1D && problem->kind != IPM_EULER_1D && problem->kind != IPM_EULER_2D)
    return "unknown problem kind";
  if (problem->kind == IPM_EULER_2D) {
    if (problem->ny < 1 || !(problem->y_hi > problem->y_lo))
      return "2-D mesh needs ny >= 1 and y_hi > y_lo";
    if ((problem->bc_bottom == IPM_BC_PERIODIC) != (problem->bc_top == IPM_BC_PERIODIC))
      return "periodic must be set on both the bottom and the top";
    const int sides[4] = {problem->bc_left, problem->bc_right, problem->bc_bottom, problem->bc_top};
    for (int k = 0; k < 4; ++k)
      if (sides[k] < IPM_BC_OUTFLOW || sides[k] > IPM_BC_SLIP_WALL) return "bad side";
    if (problem->mesh_kind != IPM_MESH_CARTESIAN && problem->mesh_kind != IPM_MESH_RAMP)
      return "unknown mesh kind";
    if (problem->mesh_kind == IPM_MESH_RAMP && !(std::fabs(problem->ramp_deg) < 60.0))
      return "ramp angle must be below 60 degrees";
    if (problem->ic_kind != IPM_IC_RIEMANN && problem->ic_kind != IPM_IC_FREESTREAM && problem->ic_kind != IPM_IC_SHEAR)
      return "unknown initial data";
    if (problem->ic_kind != IPM_IC_FREESTREAM && problem->mesh_kind != IPM_MESH_CARTESIAN)
      return "Riemann and shear data need a Cartesian mesh";
  } else if (problem->bc_left == IPM_BC_SLIP_WALL || problem->bc_right == IPM_BC_SLIP_WALL) {
    return "slip walls are 2-D only";
  }
  if (problem->nx < 1 || !(problem->x_hi > problem->x_lo) || !(problem->cfl > 0))
    return "bad mesh or cfl";
  if ((problem->bc_left == IPM_BC_PERIODIC) != (problem->bc_right == IPM_BC_PERIODIC))
    return "periodic must be set on both ends";
  return nullptr;
}
}  // namespace ipm

// Validate the problem and fill every size, table and launch parameter of c (no device allocation).
static ipm_status plan_ctx(ipm_ctx* c, const ipm_problem* problem, const ipm_basis* basis, const ipm_quadrature* quad,
                           const ipm_entropy* entropy, const ipm_options& opt) {
  if (const char* why = check_problem(problem, basis, quad)) return fail(nullptr, IPM_EINVAL, std::string("ipm_init: ") + why);
  if (opt.precision != IPM_PREC_FP64 && opt.precision != IPM_PREC_MIXED && opt.precision != IPM_PREC_MIXED_F32_FACTOR)
    return fail(nullptr, IPM_EINVAL, "ipm_init: unknown precision");
  if (opt.precision == IPM_PREC_MIXED_F32_FACTOR && opt.hessian_reuse != 0)
    return fail(nullptr, IPM_EINVAL, "ipm_init: frozen Hessians keep FP64 factors; use them with IPM_PREC_FP64 or _MIXED");
  if (opt.newton_kernel < 0 || opt.newton_kernel > 2) return fail(nullptr, IPM_EINVAL, "ipm_init: unknown Newton kernel");
  if (opt.hessian_reuse < 0 || opt.hessian_reuse > 2 || !(opt.reuse_ratio > 0.0 && opt.reuse_ratio < 1.0))
    return fail(nullptr, IPM_EINVAL, "ipm_init: hessian_reuse must be 0..2 with 0 < reuse_ratio < 1");
  if (opt.check_cache != 0 && opt.check_cache != 1) return fail(nullptr, IPM_EINVAL, "ipm_init: check_cache must be 0 or 1");
  if (opt.factorization < 0 || opt.factorization > 2) return fail(nullptr, IPM_EINVAL, "ipm_init: factorization must be 0..2");
  if (opt.factorization == 2 && opt.precision == IPM_PREC_MIXED_F32_FACTOR)
    return fail(nullptr, IPM_EINVAL, "ipm_init: the split factorisation is an FP64 factorisation; not with IPM_PREC_MIXED_F32_FACTOR");
  c->prob = *problem;
  c->basis = *basis;
  c->quad = *quad;
  c->ent = *entropy;
  c->opt = opt;
  c->is2d = problem->kind == IPM_EULER_2D;
  c->m = problem->kind == IPM_BURGERS_1D ? 1 : (c->is2d ? 4 : 3);
  c->phys = problem->kind == IPM_BURGERS_1D ? PHYS_BURGERS : (c->is2d ? PHYS_EULER2D : PHYS_EULER1D);
  c->entk = entropy->kind == IPM_ENTROPY_QUADRATIC ? ENT_QUADRATIC
                                                     : (entropy->kind == IPM_ENTROPY_BOUNDED_BARRIER ? ENT_BARRIER : ENT_EULER);
  const bool ent_ok = c->entk == ENT_QUADRATIC || (c->entk == ENT_BARRIER && c->phys == PHYS_BURGERS) ||
                      (c->entk == ENT_EULER && c->phys != PHYS_BURGERS);
  if (!ent_ok) {
    return fail(nullptr, IPM_EINVAL, "ipm_init: entropy does not match the problem");
  }
  if (c->entk == ENT_BARRIER && !(entropy->u_plus > entropy->u_minus)) {
    return fail(nullptr, IPM_EINVAL, "ipm_init: barrier needs u_plus > u_minus");
  }
  const int L_adapt = opt.adapt_min_degree > 0 ? basis->total_degree - opt.adapt_min_degree + 1 : 0;
  if (quad->kind == IPM_QUAD_CC_NESTED) {
    // nested Clenshaw-Curtis rules: one per refinement level (or one for a fixed degree)
    const int nl = L_adapt > 0 && L_adapt <= 8 ? L_adapt : 1;
    const int M0 = L_adapt > 0 ? opt.adapt_min_degree : basis->total_degree;
    int cc[8] = {0};
    if (const char* why = cc_levels(quad, M0, nl, cc)) return fail(nullptr, IPM_EINVAL, std::string("ipm_init: ") + why);
    int q1 = 1;
    for (int d = 0; d < basis->p; ++d) q1 *= (cc[nl - 1] == 0 ? 1 : (1 << cc[nl - 1]) + 1);
    if (q1 > 40000) return fail(nullptr, IPM_EINVAL, "ipm_init: the finest Clenshaw-Curtis rule has more than 40000 nodes");
    std::vector<std::vector<double>> lw;
    build_tables_cc(basis->p, basis->total_degree, cc[nl - 1], c->tab, lw);
    if (L_adapt > 0) {
      c->level_rules = true;
      c->lev_w.assign((size_t)nl * c->tab.Q, 0.0);
      for (int l = 0; l < nl; ++l) {
        c->lev_q[l] = (int)lw[cc[l]].size();
        std::copy(lw[cc[l]].begin(), lw[cc[l]].end(), c->lev_w.begin() + (size_t)l * c->tab.Q);
      }
    }
  } else {
    build_tables(basis->p, basis->total_degree, quad->n_per_dim, c->tab);
  }
  c->N = c->tab.N;
  c->Q = c->tab.Q;
  for (int l = 0; l < 8; ++l)
    if (!c->level_rules) c->lev_q[l] = c->Q;
  c->NM = c->N * c->m;
  c->n_interior = c->is2d ? problem->nx * problem->ny : problem->nx;
  c->n_cells = c->is2d ? (problem->nx + 2) * (problem->ny + 2) : problem->nx + 2;
  c->dx = (problem->x_hi - problem->x_lo) / problem->nx;
  if (c->is2d) build_mesh2d(*problem, c->mesh2d);
  if (opt.hessian_reuse == 2) {
    c->factor_stride = (size_t)c->NM * (c->NM + 1) / 2 + c->NM;
    size_t free_b = 0;
    if (available_device_bytes(&free_b) != cudaSuccess ||
        (size_t)c->n_cells * c->factor_stride * sizeof(double) > free_b / 4)
      return fail(nullptr, IPM_EINVAL, "ipm_init: kept factors (hessian_reuse 2) need more than a quarter of the free memory");
  }
  if (opt.adapt_min_degree > 0) {
    if (!c->is2d) return fail(nullptr, IPM_EINVAL, "ipm_init: adaptivity is built for 2-D problems");
    const int L = basis->total_degree - opt.adapt_min_degree + 1;
    if (L < 1 || L > 8) return fail(nullptr, IPM_EINVAL, "ipm_init: adaptivity needs 1..8 levels up to the basis degree");
    c->n_levels = L;
    for (int l = 0; l < L; ++l) {
      const int M = opt.adapt_min_degree + l;
      int n = 0, np = 0;
      for (int i = 0; i < c->N; ++i) {
        int deg = 0;
        for (int d = 0; d < c->tab.p; ++d) deg += c->tab.indices[(size_t)i * c->tab.p + d];
        n += deg <= M;
        np += deg <= M - 1;
      }
      c->lev_n[l] = n;
      c->lev_prev[l] = np;
    }
  }
  if (c->N > 65535) {
    return fail(nullptr, IPM_EINVAL, "ipm_init: too many moments");
  }

  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) {
    return fail(nullptr, IPM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  }
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, c->device);
  if (e != cudaSuccess) {
    return fail(nullptr, IPM_ECUDA, std::string("cudaGetDeviceProperties: ") + cudaGetErrorString(e));
  }
  // launch configuration of the Newton kernel: packed H in shared memory when it fits
  const size_t budget = (size_t)prop.sharedMemPerBlockOptin;
  c->mixed = opt.precision != IPM_PREC_FP64;
  // factorisation: 1 blocked FP64 FMAs; 2 split (FP64-accurate, trailing updates on the tensor cores);
  // 0 picks the split one on the mixed path for systems of at least SPLIT_AUTO_NM unknowns
  c->split = opt.factorization == 2 ||
             (opt.factorization == 0 && opt.precision == IPM_PREC_MIXED && c->NM >= SPLIT_AUTO_NM);
  c->s_rows = c->split ? split_rows(c->NM) : 0;
  c->newton_mode = opt.precision == IPM_PREC_MIXED_F32_FACTOR ? 2 : (c->mixed ? (c->split ? 3 : 1) : (c->split ? 4 : 0));
  if (c->mixed) {
    c->h_in_smem = true;
    c->mx = mixed_layout(c->N, c->m, c->Q, budget, true, c->s_rows);
    if (!c->mx.ok) {
      c->h_in_smem = false;
      c->mx = mixed_layout(c->N, c->m, c->Q, budget, false, c->s_rows);
    }
    if (!c->mx.ok && c->split && opt.factorization == 0) {
      // the digit slices do not fit next to the tensor-core Hessian: the automatic choice falls back
      c->split = false;
      c->s_rows = 0;
      c->newton_mode = 1;
      c->h_in_smem = true;
      c->mx = mixed_layout(c->N, c->m, c->Q, budget, true, 0);
      if (!c->mx.ok) {
        c->h_in_smem = false;
        c->mx = mixed_layout(c->N, c->m, c->Q, budget, false, 0);
      }
    }
    if (!c->mx.ok) {
        return fail(nullptr, IPM_EINVAL, "ipm_init: N*m and Q too large for the mixed-precision Newton kernel");
    }
    c->sm = newton_smem(c->N, c->m, c->Q, c->h_in_smem, &c->mx, c->s_rows);
    // the digit-slice region of the split factorisation is idle while the Hessian is assembled: when it
    // has a region of its own (not the A staging) it holds two staged Phi^T chunks for the A builds
    const size_t stage_bytes = 2 * (size_t)c->N * (c->mx.kc + 4) * sizeof(float);
    if (c->split && c->sm.off_s != c->sm.off_a && split_bytes(c->s_rows) >= stage_bytes) {
      c->ph_stage_off = c->sm.off_s;
    } else if (!c->split) {
      // without a digit-slice region: a staging region of its own, when the shared memory has room and
      // the CTAs resident per SM stay as many
      const size_t off = (c->sm.bytes + 127) & ~(size_t)127, with = off + stage_bytes;
      const size_t per_sm = (size_t)prop.sharedMemPerMultiprocessor, rsv = (size_t)prop.reservedSharedMemPerBlock;
      if (with + 1024 <= budget && per_sm / (with + rsv) == per_sm / (c->sm.bytes + rsv)) {
        c->ph_stage_off = (uint32_t)off;
        c->sm.bytes = with;
      }
    }
  } else {
    const NewtonSmem full = newton_smem(c->N, c->m, c->Q, true, nullptr, c->s_rows);
    const NewtonSmem lean = newton_smem(c->N, c->m, c->Q, false, nullptr, c->s_rows);
    if (lean.bytes > budget) {
        return fail(nullptr, IPM_EINVAL, "ipm_init: N*m and Q too large for one CTA");
    }
    c->h_in_smem = full.bytes <= budget;
    c->sm = c->h_in_smem ? full : lean;
    if (c->split) c->mx.tmem_cols = SPLIT_TMEM_COLS_ONE;
  }
  c->newton_smem = c->sm.bytes;
  {
    // persistent grid: resident CTAs per SM (occupancy API) times the SM count; on the mixed path
    // the CTAs of one SM must also share its 512 tensor-memory columns
    int bps = 0;
    e = prepare_newton(c->entk, c->phys, c->m, c->newton_smem, c->h_in_smem, c->newton_mode, &bps);
    if (e == cudaSuccess) e = c->is2d ? prepare_update2d(c->N, c->Q) : prepare_update1d(c->phys, c->m, c->N, c->Q);
    if (e != cudaSuccess || bps < 1) {
        return fail(nullptr, IPM_ECUDA, std::string("kernel set-up: ") + cudaGetErrorString(e));
    }
    if (c->split) {
      // two accumulator sets (MMAs of the next unit overlap the combine of this one) when one CTA per
      // SM is resident anyway, or when the Hessian already holds all 512 columns
      if (bps == 1) c->mx.tmem_cols = 512;
      else c->mx.tmem_cols = std::max(c->mx.tmem_cols, SPLIT_TMEM_COLS_ONE);
      c->s_nbuf = c->mx.tmem_cols >= 2 * SPLIT_TMEM_COLS_ONE ? 2 : 1;
    }
    if (c->mixed || c->split) bps = std::min(bps, 512 / c->mx.tmem_cols);
    c->newton_grid = std::max(1, std::min(c->n_interior, bps * prop.multiProcessorCount));
  }
  // warp-per-cell variant for small cells: as many warps (cells) per CTA as shared memory allows
  if (c->NM <= 64 && c->n_levels == 0 && opt.hessian_reuse == 0 && c->newton_mode != 2) {
    const size_t slice = newton_warp_slice(c->N, c->m, c->Q);
    for (int wps = 8; wps >= 2; wps /= 2) {
      if (wps * slice * sizeof(double) > budget) continue;
      int bps = 0;
      if (prepare_newton_warp(c->entk, c->phys, c->m, c->mixed, wps, (int)slice, &bps) == cudaSuccess && bps >= 1) {
        c->warp_warps = wps;
        c->warp_slice = (int)slice;
        c->warp_grid = bps * prop.multiProcessorCount;
        break;
      }
    }
  }
  // adaptive meshes: the lowest levels with N m <= 64 go to the warp-per-cell kernel (Newton iterations
  // and the mixed Hessian as in the warp kernel, an FP64 factorisation of these small systems in every
  // precision mode); frozen Hessians keep the CTA kernel, as does newton_kernel = 1
  if (c->n_levels > 0 && opt.hessian_reuse == 0 && opt.newton_kernel != 1) {
    int L = 0;
    while (L < c->n_levels && c->lev_n[L] * c->m <= 64) ++L;
    if (L > 0) {
      const int nm = c->lev_n[L - 1] * c->m;
      const size_t slice = newton_warpq_slice(nm, c->m);
      for (int wps = 8; wps >= 1; wps /= 2) {
        if (wps * slice * sizeof(double) > budget) continue;
        int bps = 0;
        if (prepare_newton_warpq(c->entk, c->phys, c->m, c->mixed, wps, (int)slice, &bps) == cudaSuccess && bps >= 1) {
          c->warp_levels = L;
          c->wq_warps = wps;
          c->wq_slice = (int)slice;
          c->wq_nm = nm;
          c->wq_grid = bps * prop.multiProcessorCount;
          break;
        }
      }
      cudaGetLastError();
    }
  }
  c->hwork_stride = c->h_in_smem ? 0 : packed_aug_count(c->NM);
  c->update_grid = std::min(c->n_interior, 65535);
  // moment images: fixed degree, or adaptive degree on one rule for every level (with a rule per level
  // the nodal states a cell writes depend on its neighbours' levels too)
  c->img = opt.check_cache != 0 && !c->level_rules;
  return IPM_OK;
}

// Device bytes ipm_init allocates for a planned context.
static size_t ctx_footprint(const ipm_ctx* c) {
  const size_t Q = c->Q, N = c->N, nc = c->n_cells, NM = c->NM;
  size_t b = 2 * Q * N * 8 + Q * 8 + Q * c->tab.p * 8 + (N * (N + 1) / 2) * 4;   // tables
  b += 2 * nc * NM * 8 + nc * c->m * Q * 8 + nc * 8 + 3 * nc * 4 + sizeof(StepScalars);
  if (!c->h_in_smem) b += (size_t)c->newton_grid * c->hwork_stride * 8;
  if (c->mixed) b += N * Q * 4 + (size_t)c->mx.chunks * (c->mx.b_chunk_bytes + N * (c->mx.kc + 4) * 4);
  if (c->is2d) b += (c->mesh2d.area.size() + c->mesh2d.xf.size() + c->mesh2d.yf.size()) * 8;
  if (c->n_levels) b += 2 * nc * 4;
  if (c->level_rules) b += nc * 4 + c->lev_w.size() * 8;
  if (c->factor_stride) b += nc * (c->factor_stride * 8 + 4);
  if (c->img) b += nc * (2 * NM * 8 + 8 + 4);
  if (!c->is2d) b += nc * (2 * NM * 8 + 4);
  return b;
}

extern "C" {

void ipm_default_options(ipm_options* o) {
  if (!o) return;
  o->precision = IPM_PREC_FP64;
  o->newton_tol = 1e-10;
  o->max_newton = 100;
  o->armijo_c = 1e-4;
  o->max_halvings = 30;
  o->slack_rel = 1e-12;
  o->adapt_min_degree = 0;
  o->delta_lo = 2e-5;
  o->delta_hi = 2e-4;
  o->hessian_reuse = 0;
  o->reuse_ratio = 0.5;
  o->newton_kernel = 0;
  o->check_cache = 1;
  o->factorization = 0;
}

const char* ipm_last_error(const ipm_ctx* c) {
  if (c) return c->err.c_str();
  std::lock_guard<std::mutex> lk(g_err_mu);
  return g_init_err.c_str();
}

ipm_status ipm_tables(int p, int total_degree, int n_per_dim, int N_cap, int Q_cap, int* indices, double* nodes,
                      double* weights, double* phi, int* N_out, int* Q_out) {
  if (p < 1 || p > 3 || total_degree < 0 || n_per_dim < 1) return fail(nullptr, IPM_EINVAL, "ipm_tables: bad sizes");
  HostTables t;
  build_tables(p, total_degree, n_per_dim, t);
  if (N_out) *N_out = t.N;
  if (Q_out) *Q_out = t.Q;
  if (t.N > N_cap || t.Q > Q_cap) return fail(nullptr, IPM_EINVAL, "ipm_tables: capacity too small");
  if (indices) std::memcpy(indices, t.indices.data(), t.indices.size() * sizeof(int));
  if (nodes) std::memcpy(nodes, t.nodes.data(), t.nodes.size() * sizeof(double));
  if (weights) std::memcpy(weights, t.w.data(), t.w.size() * sizeof(double));
  if (phi) std::memcpy(phi, t.Phi.data(), t.Phi.size() * sizeof(double));
  return IPM_OK;
}

ipm_status ipm_tables_cc(int p, int total_degree, int kmax, int N_cap, int Q_cap, int* indices, double* nodes,
                         double* level_weights, double* phi, int* N_out, int* Q_out) {
  if (p < 1 || p > 3 || total_degree < 0 || kmax < 0 || kmax > 6) return fail(nullptr, IPM_EINVAL, "ipm_tables_cc: bad sizes");
  HostTables t;
  std::vector<std::vector<double>> lw;
  build_tables_cc(p, total_degree, kmax, t, lw);
  if (N_out) *N_out = t.N;
  if (Q_out) *Q_out = t.Q;
  if (t.N > N_cap || t.Q > Q_cap) return fail(nullptr, IPM_EINVAL, "ipm_tables_cc: capacity too small");
  if (indices) std::memcpy(indices, t.indices.data(), t.indices.size() * sizeof(int));
  if (nodes) std::memcpy(nodes, t.nodes.data(), t.nodes.size() * sizeof(double));
  if (level_weights)
    for (int k = 0; k <= kmax; ++k)
      for (int q = 0; q < t.Q; ++q) level_weights[(size_t)k * t.Q + q] = q < (int)lw[k].size() ? lw[k][q] : 0.0;
  if (phi) std::memcpy(phi, t.Phi.data(), t.Phi.size() * sizeof(double));
  return IPM_OK;
}

ipm_status ipm_footprint(const ipm_problem* problem, const ipm_basis* basis, const ipm_quadrature* quad,
                         const ipm_entropy* entropy, const ipm_options* options, size_t* bytes) {
  if (!problem || !basis || !quad || !entropy || !bytes) return fail(nullptr, IPM_EINVAL, "ipm_footprint: NULL argument");
  ipm_options opt;
  if (options) opt = *options;
  else ipm_default_options(&opt);
  ipm_ctx c;
  const ipm_status st = plan_ctx(&c, problem, basis, quad, entropy, opt);
  if (st != IPM_OK) return st;
  *bytes = ctx_footprint(&c);
  return IPM_OK;
}

ipm_status ipm_init(const ipm_problem* problem, const ipm_basis* basis, const ipm_quadrature* quad,
                    const ipm_entropy* entropy, const ipm_options* options, ipm_ctx** out) {
  NvtxRange nvtx_("ipm_init");
  if (!problem || !basis || !quad || !entropy || !out) return fail(nullptr, IPM_EINVAL, "ipm_init: NULL argument");
  *out = nullptr;
  ipm_options opt;
  if (options) opt = *options;
  else ipm_default_options(&opt);

  ipm_ctx* c = new ipm_ctx();
  {
    const ipm_status ps = plan_ctx(c, problem, basis, quad, entropy, opt);
    if (ps != IPM_OK) {
      delete c;
      return ps;
    }
  }
  cudaError_t e = cudaSuccess;

  ipm_status st = IPM_OK;
  auto CK = [&](cudaError_t err, const char* what) {
    if (err != cudaSuccess) cudaGetLastError();          // clear a non-sticky error for later launches
    if (err != cudaSuccess && st == IPM_OK) {
      st = fail(nullptr, err == cudaErrorMemoryAllocation ? IPM_ENOMEM : IPM_ECUDA,
                std::string(what) + ": " + cudaGetErrorString(err));
    }
  };
  CK(cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking), "cudaStreamCreate");
  for (cudaEvent_t& ev : c->ev) CK(cudaEventCreate(&ev), "cudaEventCreate");
  c->stream = c->own_stream;
  CK(upload(c, &c->d_Phi, c->tab.Phi), "upload Phi");
  CK(upload(c, &c->d_PhiT, c->tab.PhiT), "upload PhiT");
  CK(upload(c, &c->d_w, c->tab.w), "upload w");
  CK(upload(c, &c->d_nodes, c->tab.nodes), "upload nodes");
  CK(upload(c, &c->d_pairs, c->tab.pairs), "upload pairs");
  if (c->mixed) {
    CK(dalloc(c, &c->d_phiT32, (size_t)c->N * c->Q * sizeof(float)), "allocate phiT32");
    CK(dalloc(c, &c->d_phi32c, (size_t)c->mx.chunks * c->N * (c->mx.kc + 4) * sizeof(float)), "allocate phi32c");
    CK(dalloc(c, &c->d_phi_img, (size_t)c->mx.chunks * c->mx.b_chunk_bytes), "allocate phi image");
    if (st == IPM_OK)
      CK(launch_phi_images(c->d_PhiT, c->N, c->Q, c->mx, c->d_phiT32, c->d_phi32c, c->d_phi_img, c->stream),
         "phi images");
  }
  const size_t nstate = (size_t)c->n_cells * c->NM;
  CK(dalloc(c, &c->d_uhat, nstate * sizeof(double)), "allocate uhat");
  CK(dalloc(c, &c->d_lam, nstate * sizeof(double)), "allocate lam");
  CK(dalloc(c, &c->d_unode, (size_t)c->n_cells * c->m * c->Q * sizeof(double)), "allocate unode");
  CK(dalloc(c, &c->d_cell_resid, (size_t)c->n_cells * sizeof(double)), "allocate resid");
  CK(dalloc(c, &c->d_iters, (size_t)c->n_cells * sizeof(int)), "allocate iters");
  CK(dalloc(c, &c->d_status, (size_t)c->n_cells * sizeof(int)), "allocate status");
  CK(dalloc(c, &c->d_order, (size_t)c->n_interior * sizeof(int)), "allocate order");
  CK(dalloc(c, &c->d_sc, sizeof(StepScalars)), "allocate scalars");
  if (!c->h_in_smem) CK(dalloc(c, &c->d_hwork, (size_t)c->newton_grid * c->hwork_stride * sizeof(double)), "allocate hwork");
  if (c->factor_stride) {
    CK(dalloc(c, &c->d_factors, (size_t)c->n_cells * c->factor_stride * sizeof(double)), "allocate factors");
    CK(dalloc(c, &c->d_factor_valid, (size_t)c->n_cells * sizeof(int)), "allocate factor flags");
    if (st == IPM_OK) CK(cudaMemsetAsync(c->d_factor_valid, 0, (size_t)c->n_cells * sizeof(int), c->stream), "memset factor flags");
  }
  if (c->img) {
    CK(dalloc(c, &c->d_img, nstate * sizeof(double)), "allocate moment images");
    CK(dalloc(c, &c->d_img_lam, nstate * sizeof(double)), "allocate image duals");
    CK(dalloc(c, &c->d_img_smax, (size_t)c->n_cells * sizeof(double)), "allocate image speeds");
    CK(dalloc(c, &c->d_img_valid, (size_t)c->n_cells * sizeof(int)), "allocate image flags");
    if (st == IPM_OK) CK(cudaMemsetAsync(c->d_img_valid, 0, (size_t)c->n_cells * sizeof(int), c->stream), "memset image flags");
  }
  if (!c->is2d) {
    CK(dalloc(c, &c->d_lf_a, nstate * sizeof(double)), "allocate folded update terms");
    CK(dalloc(c, &c->d_lf_b, nstate * sizeof(double)), "allocate folded update terms");
    CK(dalloc(c, &c->d_lf_cnt, (size_t)c->n_cells * sizeof(int)), "allocate folded update counts");
  }
  if (st != IPM_OK) {
    free_ctx(c);
    return st;
  }
  CK(cudaMemsetAsync(c->d_sc, 0, sizeof(StepScalars), c->stream), "memset scalars");
  CK(cudaMemsetAsync(c->d_iters, 0, (size_t)c->n_cells * sizeof(int), c->stream), "memset iters");
  CK(cudaMemsetAsync(c->d_status, 0, (size_t)c->n_cells * sizeof(int), c->stream), "memset status");
  CK(cudaMemsetAsync(c->d_cell_resid, 0, (size_t)c->n_cells * sizeof(double), c->stream), "memset resid");
  CK(cudaMemsetAsync(c->d_unode, 0, (size_t)c->n_cells * c->m * c->Q * sizeof(double), c->stream), "memset unode");
  // initial data on every cell, then the boundary copies (1-D) or the mesh tables (2-D)
  if (c->is2d) {
    CK(upload(c, &c->d_area, c->mesh2d.area), "upload areas");
    CK(upload(c, &c->d_xf, c->mesh2d.xf), "upload x faces");
    CK(upload(c, &c->d_yf, c->mesh2d.yf), "upload y faces");
    if (st == IPM_OK)
      CK(launch_init2d(c->entk, dev_tables(c), ent_params(c), c->prob, c->d_uhat, c->d_lam, c->stream), "init kernel");
    if (c->n_levels) {
      CK(dalloc(c, &c->d_level, (size_t)c->n_cells * sizeof(int)), "allocate levels");
      CK(dalloc(c, &c->d_level_next, (size_t)c->n_cells * sizeof(int)), "allocate next levels");
      if (c->level_rules) {
        CK(upload(c, &c->d_lev_w, c->lev_w), "upload level weights");
        CK(upload(c, &c->d_q_eval, std::vector<int>((size_t)c->n_cells, c->Q)), "upload evaluation nodes");
      }
      if (st == IPM_OK)
        CK(launch_init_levels(update2d_args(c, 0.0, false, false), c->n_cells, c->stream), "initial levels");
      // with a rule per level, every cell's initial moments and duals come from its level's rule
      if (st == IPM_OK && c->level_rules)
        CK(launch_init2d(c->entk, dev_tables(c), ent_params(c), c->prob, c->d_uhat, c->d_lam, c->stream, c->d_level,
                         c->lev_n, c->lev_q, c->d_lev_w),
           "initial data at the level rules");
      if (st == IPM_OK)
        CK(cudaMemcpyAsync(c->d_level_next, c->d_level, (size_t)c->n_cells * sizeof(int), cudaMemcpyDeviceToDevice,
                           c->stream),
           "copy levels");
    }
  } else {
    CK(launch_init1d(c->entk, c->m, dev_tables(c), ent_params(c), c->prob, c->d_uhat, c->d_lam, c->n_cells, c->stream),
       "init kernel");
    CK(launch_bc_copy1d(c->d_uhat, c->d_lam, problem->nx, c->NM, problem->bc_left, problem->bc_right, c->stream),
       "bc kernel");
  }
  // Dirichlet ghosts: converge their duals once; their speed stays part of every dt
  std::vector<int> ghosts;
  if (c->is2d) {
    const int nx = problem->nx, ny = problem->ny;
    auto cell = [&](int i, int j) { return (j + 1) * (nx + 2) + (i + 1); };
    for (int j = 0; j < ny; ++j) {
      if (problem->bc_left == IPM_BC_DIRICHLET) ghosts.push_back(cell(-1, j));
      if (problem->bc_right == IPM_BC_DIRICHLET) ghosts.push_back(cell(nx, j));
    }
    for (int i = 0; i < nx; ++i) {
      if (problem->bc_bottom == IPM_BC_DIRICHLET) ghosts.push_back(cell(i, -1));
      if (problem->bc_top == IPM_BC_DIRICHLET) ghosts.push_back(cell(i, ny));
    }
  } else {
    if (problem->bc_left == IPM_BC_DIRICHLET) ghosts.push_back(0);
    if (problem->bc_right == IPM_BC_DIRICHLET) ghosts.push_back(problem->nx + 1);
  }
  c->n_fixed_ghosts = (int)ghosts.size();
  if (!ghosts.empty()) {
    CK(upload(c, &c->d_ghost_list, ghosts), "upload ghosts");
    if (st == IPM_OK) {
      NewtonArgs a = newton_args(c, 0);
      a.cell_list = c->d_ghost_list;
      a.n_work = (int)ghosts.size();
      CK(launch_newton_ctx(c, a, (int)ghosts.size(), c->stream), "ghost solve");
    }
  }
  if (st == IPM_OK) {
    // fixed speed = what the ghost solve folded in (0 without Dirichlet ghosts); then reset counters
    StepScalars h;
    std::vector<int> status(c->n_cells, 0);
    CK(cudaMemcpyAsync(&h, c->d_sc, sizeof(StepScalars), cudaMemcpyDeviceToHost, c->stream), "read scalars");
    CK(cudaMemcpyAsync(status.data(), c->d_status, status.size() * sizeof(int), cudaMemcpyDeviceToHost, c->stream),
       "read ghost status");
    CK(cudaStreamSynchronize(c->stream), "init sync");
    if (st == IPM_OK) {
      for (int g : ghosts)
        if (status[g] != 0) st = fail(nullptr, IPM_EINVAL, "ipm_init: Dirichlet ghost dual solve failed");
      h.fixed_smax_bits = h.smax_bits;
      h.level_cap = c->n_levels ? c->n_levels - 1 : 0;
      h.work_counter = 0;
      h.update_counter = 0;
      h.t = 0.0;
      h.dt = 0.0;
      h.steps = 0;
      CK(cudaMemcpyAsync(c->d_sc, &h, sizeof(StepScalars), cudaMemcpyHostToDevice, c->own_stream), "write scalars");
      // per-cell counters start from zero (the step reductions of 2-D meshes include the ghosts)
      CK(cudaMemsetAsync(c->d_iters, 0, (size_t)c->n_cells * sizeof(int), c->own_stream), "reset iters");
    }
  }
  if (st == IPM_OK && c->warp_warps > 0) {
    if (c->opt.newton_kernel == 0) st = autotune_newton(c);
    else c->newton_kind = c->opt.newton_kernel == 2 ? 1 : 0;
    // the timing runs restored the duals but left images and nodal states of their own
    if (st == IPM_OK && c->img)
      CK(cudaMemsetAsync(c->d_img_valid, 0, (size_t)c->n_cells * sizeof(int), c->stream), "reset image flags");
  } else if (st == IPM_OK && c->opt.newton_kernel == 2) {
    st = fail(nullptr, IPM_EINVAL, "ipm_init: the warp-per-cell kernel needs N*m <= 64 and a fixed degree");
  }
  if (st == IPM_OK) st = build_graph(c, 0, &c->step_exec);
  if (st == IPM_OK) st = build_graph(c, 1, &c->oneshot_exec);
  if (st != IPM_OK) {
    if (!c->err.empty()) fail(nullptr, st, c->err);
    free_ctx(c);
    return st;
  }
  *out = c;
  return IPM_OK;
}

void ipm_destroy(ipm_ctx* c) {
  if (c && c->stream) cudaStreamSynchronize(c->stream);
  free_ctx(c);
}

ipm_status ipm_get_dims(const ipm_ctx* c, ipm_dims* d) {
  if (!c || !d) return IPM_EINVAL;
  d->N = c->N;
  d->m = c->m;
  d->Q = c->Q;
  d->p = c->tab.p;
  d->n_cells = c->n_cells;
  d->n_interior = c->n_interior;
  return IPM_OK;
}

ipm_status ipm_set_stream(ipm_ctx* c, void* s) {
  if (!c) return IPM_EINVAL;
  IPM_CK(c, cudaStreamSynchronize(c->stream));
  c->stream = static_cast<cudaStream_t>(s);
  return IPM_OK;
}

static ipm_status copy_state(ipm_ctx* c, void* dst, const void* src, size_t count, size_t expect, cudaMemcpyKind kind,
                             bool sync) {
  if (!c || (!dst && count) || (!src && count)) return fail(c, IPM_EINVAL, "copy: NULL pointer");
  if (count != expect) return fail(c, IPM_EINVAL, "copy: count does not match the state size");
  IPM_CK(c, cudaMemcpyAsync(dst, src, count * sizeof(double), kind, c->stream));
  if (sync) IPM_CK(c, cudaStreamSynchronize(c->stream));
  return IPM_OK;
}

ipm_status ipm_set_moments(ipm_ctx* c, const double* h, size_t n) {
  if (!c) return IPM_EINVAL;
  return copy_state(c, c->d_uhat, h, n, (size_t)c->n_cells * c->NM, cudaMemcpyHostToDevice, true);
}
ipm_status ipm_get_moments(ipm_ctx* c, double* h, size_t n) {
  if (!c) return IPM_EINVAL;
  return copy_state(c, h, c->d_uhat, n, (size_t)c->n_cells * c->NM, cudaMemcpyDeviceToHost, true);
}
ipm_status ipm_set_duals(ipm_ctx* c, const double* h, size_t n) {
  if (!c) return IPM_EINVAL;
  return copy_state(c, c->d_lam, h, n, (size_t)c->n_cells * c->NM, cudaMemcpyHostToDevice, true);
}
ipm_status ipm_get_duals(ipm_ctx* c, double* h, size_t n) {
  if (!c) return IPM_EINVAL;
  return copy_state(c, h, c->d_lam, n, (size_t)c->n_cells * c->NM, cudaMemcpyDeviceToHost, true);
}
ipm_status ipm_set_state(ipm_ctx* c, const double* mom, const double* duals, const int* levels,
                         const ipm_clock* clock, size_t n) {
  if (!c) return IPM_EINVAL;
  const size_t expect = (size_t)c->n_cells * c->NM;
  ipm_status st = copy_state(c, c->d_uhat, mom, n, expect, cudaMemcpyHostToDevice, false);
  if (st == IPM_OK) st = copy_state(c, c->d_lam, duals, n, expect, cudaMemcpyHostToDevice, false);
  if (st != IPM_OK) return st;
  if (levels && c->n_levels) {
    for (int k = 0; k < c->n_cells; ++k)
      if (levels[k] < 0 || levels[k] >= c->n_levels) return fail(c, IPM_EINVAL, "ipm_set_state: level out of range");
    IPM_CK(c, cudaMemcpyAsync(c->d_level, levels, (size_t)c->n_cells * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    IPM_CK(c, cudaMemcpyAsync(c->d_level_next, c->d_level, (size_t)c->n_cells * sizeof(int), cudaMemcpyDeviceToDevice,
                              c->stream));
  }
  if (clock) {
    if (c->n_levels && (clock->level_cap < 0 || clock->level_cap >= c->n_levels))
      return fail(c, IPM_EINVAL, "ipm_set_state: level cap out of range");
    StepScalars h;
    IPM_CK(c, cudaMemcpyAsync(&h, c->d_sc, sizeof(StepScalars), cudaMemcpyDeviceToHost, c->stream));
    IPM_CK(c, cudaStreamSynchronize(c->stream));
    h.t = clock->t;
    h.dt = clock->dt;
    h.steps = clock->steps;
    h.level_cap = c->n_levels ? clock->level_cap : 0;
    IPM_CK(c, cudaMemcpyAsync(c->d_sc, &h, sizeof(StepScalars), cudaMemcpyHostToDevice, c->stream));
  }
  IPM_CK(c, cudaStreamSynchronize(c->stream));
  return IPM_OK;
}

ipm_status ipm_get_state(ipm_ctx* c, double* mom, double* duals, int* levels, ipm_clock* clock, size_t n) {
  if (!c) return IPM_EINVAL;
  const size_t expect = (size_t)c->n_cells * c->NM;
  ipm_status st = copy_state(c, mom, c->d_uhat, n, expect, cudaMemcpyDeviceToHost, false);
  if (st == IPM_OK) st = copy_state(c, duals, c->d_lam, n, expect, cudaMemcpyDeviceToHost, false);
  if (st != IPM_OK) return st;
  if (levels && c->n_levels)
    IPM_CK(c, cudaMemcpyAsync(levels, c->d_level, (size_t)c->n_cells * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  StepScalars h;
  if (clock) IPM_CK(c, cudaMemcpyAsync(&h, c->d_sc, sizeof(StepScalars), cudaMemcpyDeviceToHost, c->stream));
  IPM_CK(c, cudaStreamSynchronize(c->stream));
  if (clock) {
    clock->t = h.t;
    clock->dt = h.dt;
    clock->steps = h.steps;
    clock->level_cap = h.level_cap;
  }
  return IPM_OK;
}

ipm_status ipm_get_nodal_states(ipm_ctx* c, double* h, size_t n) {
  if (!c) return IPM_EINVAL;
  return copy_state(c, h, c->d_unode, n, (size_t)c->n_cells * c->m * c->Q, cudaMemcpyDeviceToHost, true);
}
ipm_status ipm_set_max_level(ipm_ctx* c, int max_level) {
  if (!c) return IPM_EINVAL;
  if (!c->n_levels) return fail(c, IPM_EINVAL, "ipm_set_max_level: the context is not adaptive");
  if (max_level < 0 || max_level >= c->n_levels) return fail(c, IPM_EINVAL, "ipm_set_max_level: level out of range");
  IPM_CK(c, cudaMemcpyAsync(&c->d_sc->level_cap, &max_level, sizeof(int), cudaMemcpyHostToDevice, c->stream));
  IPM_CK(c, launch_cap_levels(update2d_args(c, 0.0, false, false), max_level, c->stream));
  IPM_CK(c, cudaStreamSynchronize(c->stream));
  return IPM_OK;
}

ipm_status ipm_oneshot_retarded(ipm_ctx* c, const int* max_levels, const double* tolerances, int n_stages, double tol,
                                int64_t max_steps, ipm_stats* s) {
  NvtxRange nvtx_("ipm_oneshot_retarded");
  if (!c || !max_levels || n_stages < 1 || (n_stages > 1 && !tolerances)) return IPM_EINVAL;
  int stage = 0;
  ipm_status st = ipm_set_max_level(c, max_levels[0]);
  if (st != IPM_OK) return st;
  ipm_stats cur;
  std::memset(&cur, 0, sizeof(cur));
  for (int64_t n = 0; n < max_steps; ++n) {
    st = ipm_oneshot_step(c, &cur);
    if (st != IPM_OK) return st;
    if (cur.failed_cells) break;
    if (stage + 1 < n_stages && cur.residual < tolerances[stage]) {
      ++stage;
      st = ipm_set_max_level(c, max_levels[stage]);
      if (st != IPM_OK) return st;
    } else if (stage + 1 == n_stages && cur.residual < tol) {
      break;
    }
  }
  if (s) *s = cur;
  return IPM_OK;
}

ipm_status ipm_get_tuning(const ipm_ctx* c, int* kernel, float* ms_cta, float* ms_warp) {
  if (!c) return IPM_EINVAL;
  if (kernel) *kernel = c->newton_kind == 1 ? 2 : 1;
  if (ms_cta) *ms_cta = c->tune_ms[0];
  if (ms_warp) *ms_warp = c->tune_ms[1];
  return IPM_OK;
}

ipm_status ipm_get_levels(ipm_ctx* c, int* h, size_t n) {
  if (!c || !h) return IPM_EINVAL;
  if (!c->n_levels) return fail(c, IPM_EINVAL, "ipm_get_levels: the context is not adaptive");
  if (n != (size_t)c->n_cells) return fail(c, IPM_EINVAL, "ipm_get_levels: count must be n_cells");
  IPM_CK(c, cudaMemcpyAsync(h, c->d_level, n * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  IPM_CK(c, cudaStreamSynchronize(c->stream));
  return IPM_OK;
}

ipm_status ipm_set_moments_device(ipm_ctx* c, const double* d, size_t n) {
  if (!c) return IPM_EINVAL;
  return copy_state(c, c->d_uhat, d, n, (size_t)c->n_cells * c->NM, cudaMemcpyDeviceToDevice, false);
}
ipm_status ipm_get_moments_device(ipm_ctx* c, double* d, size_t n) {
  if (!c) return IPM_EINVAL;
  return copy_state(c, d, c->d_uhat, n, (size_t)c->n_cells * c->NM, cudaMemcpyDeviceToDevice, false);
}

static void fill_stats(const StepScalars& h, ipm_stats* s) {
  s->newton_iters = h.newton_iters;
  s->max_iters = h.max_iters;
  s->failed_cells = h.failed_cells;
  s->first_failed_cell = h.first_failed_cell;
  s->first_status = h.first_status;
  s->dt = h.dt;
  s->t = h.t;
  s->residual = h.residual;
  s->steps = h.steps;
  s->tc_timeouts = h.tc_timeouts;
  s->factorizations = (int64_t)h.last_factorizations;
  s->fp32_fallbacks = h.fp32_fallbacks;
  s->cached_checks = (int64_t)h.last_cached_checks;
  s->hessian_ns = (int64_t)h.last_hessian_ns;
  s->hessian_count = (int64_t)h.last_hessian_count;
}

ipm_status ipm_sync_stats(ipm_ctx* c, ipm_stats* s) {
  if (!c || !s) return IPM_EINVAL;
  StepScalars h;
  IPM_CK(c, cudaMemcpyAsync(&h, c->d_sc, sizeof(StepScalars), cudaMemcpyDeviceToHost, c->stream));
  IPM_CK(c, cudaStreamSynchronize(c->stream));
  fill_stats(h, s);
  if (h.tc_stuck) {
    c->unusable = true;
    return fail(c, IPM_ETIMEOUT, "tensor-core work could not be drained after a timeout; the context is unusable");
  }
  return IPM_OK;
}

ipm_status ipm_dual_solve(ipm_ctx* c, ipm_stats* s) {
  NvtxRange nvtx_("ipm_dual_solve");
  if (!c) return IPM_EINVAL;
  if (c->unusable) return fail(c, IPM_ETIMEOUT, "context unusable after an undrained tensor-core timeout");
  IPM_CK(c, enqueue_newton(c, 0, c->stream));
  IPM_CK(c, launch_finalize(c->d_sc, c->d_iters, c->d_status, nullptr, c->n_cells, c->is2d ? 0 : 1,
                            c->is2d ? c->n_cells : c->n_interior, 0, c->stream));
  if (s) return ipm_sync_stats(c, s);
  return IPM_OK;
}

ipm_status ipm_assemble_hessian(ipm_ctx* c, double* h, size_t count) {
  NvtxRange nvtx_("ipm_assemble_hessian");
  if (!c || (!h && count)) return IPM_EINVAL;
  if (c->unusable) return fail(c, IPM_ETIMEOUT, "context unusable after an undrained tensor-core timeout");
  const size_t nph = (size_t)c->NM * (c->NM + 1) / 2;
  if (count != (size_t)c->n_interior * nph) return fail(c, IPM_EINVAL, "ipm_assemble_hessian: count must be n_interior*NM(NM+1)/2");
  double* d = nullptr;
  IPM_CK(c, dalloc(c, &d, count * sizeof(double), c->stream));
  NewtonArgs a = newton_args(c, 0);
  a.h_dump = d;
  a.track_speed = 0;
  cudaError_t e = cudaMemsetAsync(&c->d_sc->work_counter, 0, sizeof(int), c->stream);
  if (e == cudaSuccess)
    e = launch_newton_phys(c->entk, c->phys, c->m, a, c->newton_grid, c->newton_smem, c->h_in_smem, c->newton_mode,
                           c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(&c->d_sc->work_counter, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, count * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFreeAsync(d, c->stream);
  IPM_CK(c, e);
  return IPM_OK;
}

ipm_status ipm_factor_hessian(ipm_ctx* c, double* h, size_t count) {
  NvtxRange nvtx_("ipm_factor_hessian");
  if (!c || (!h && count)) return IPM_EINVAL;
  if (c->unusable) return fail(c, IPM_ETIMEOUT, "context unusable after an undrained tensor-core timeout");
  const size_t nph = (size_t)c->NM * (c->NM + 1) / 2;
  if (count != (size_t)c->n_interior * nph) return fail(c, IPM_EINVAL, "ipm_factor_hessian: count must be n_interior*NM(NM+1)/2");
  double* d = nullptr;
  IPM_CK(c, dalloc(c, &d, count * sizeof(double), c->stream));
  NewtonArgs a = newton_args(c, 0);
  a.f_dump = d;
  a.track_speed = 0;
  cudaError_t e = cudaMemsetAsync(&c->d_sc->work_counter, 0, sizeof(int), c->stream);
  if (e == cudaSuccess)
    e = launch_newton_phys(c->entk, c->phys, c->m, a, c->newton_grid, c->newton_smem, c->h_in_smem, c->newton_mode,
                           c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(&c->d_sc->work_counter, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, count * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFreeAsync(d, c->stream);
  IPM_CK(c, e);
  return IPM_OK;
}

ipm_status ipm_update(ipm_ctx* c, double dt) {
  NvtxRange nvtx_("ipm_update");
  if (!c) return IPM_EINVAL;
  if (c->unusable) return fail(c, IPM_ETIMEOUT, "context unusable after an undrained tensor-core timeout");
  if (!(dt > 0.0)) return fail(c, IPM_EINVAL, "ipm_update: dt must be positive");
  if (c->is2d) {
    IPM_CK(c, launch_update2d(update2d_args(c, dt, false, false), c->update_grid, c->stream));
  } else {
    Update1DArgs u = update_args(c, dt, false);
    IPM_CK(c, launch_update1d(c->phys, c->m, u, c->update_grid, c->stream));
  }
  IPM_CK(c, cudaStreamSynchronize(c->stream));
  return IPM_OK;
}

ipm_status ipm_step(ipm_ctx* c, ipm_stats* s) {
  NvtxRange nvtx_("ipm_step");
  if (!c) return IPM_EINVAL;
  if (c->unusable) return fail(c, IPM_ETIMEOUT, "context unusable after an undrained tensor-core timeout");
  IPM_CK(c, cudaGraphLaunch(c->step_exec, c->stream));
  if (s) return ipm_sync_stats(c, s);
  return IPM_OK;
}

ipm_status ipm_oneshot_step(ipm_ctx* c, ipm_stats* s) {
  NvtxRange nvtx_("ipm_oneshot_step");
  if (!c) return IPM_EINVAL;
  if (c->unusable) return fail(c, IPM_ETIMEOUT, "context unusable after an undrained tensor-core timeout");
  IPM_CK(c, cudaGraphLaunch(c->oneshot_exec, c->stream));
  if (s) return ipm_sync_stats(c, s);
  return IPM_OK;
}

ipm_status ipm_step_timing(ipm_ctx* c, float* newton_ms, float* update_ms, float* total_ms) {
  if (!c) return IPM_EINVAL;
  IPM_CK(c, cudaEventSynchronize(c->ev[3]));
  float a = 0.f, b = 0.f, t = 0.f;
  IPM_CK(c, cudaEventElapsedTime(&a, c->ev[0], c->ev[1]));
  IPM_CK(c, cudaEventElapsedTime(&b, c->ev[1], c->ev[2]));
  IPM_CK(c, cudaEventElapsedTime(&t, c->ev[0], c->ev[3]));
  if (newton_ms) *newton_ms = a;
  if (update_ms) *update_ms = b;
  if (total_ms) *total_ms = t;
  return IPM_OK;
}

ipm_status ipm_run(ipm_ctx* c, int64_t max_steps, ipm_stats* s) {
  NvtxRange nvtx_("ipm_run");
  if (!c) return IPM_EINVAL;
  if (c->unusable) return fail(c, IPM_ETIMEOUT, "context unusable after an undrained tensor-core timeout");
  if (!(c->prob.t_end > 0.0)) return fail(c, IPM_EINVAL, "ipm_run: t_end must be positive");
  ipm_stats cur;
  ipm_status st = ipm_sync_stats(c, &cur);
  if (st != IPM_OK) return st;
  int64_t done = 0;
  while (cur.t < c->prob.t_end && done < max_steps) {
    // launch a batch sized from the last dt; extra launches after t_end are no-ops on the device
    int64_t batch = 16;
    if (cur.dt > 0.0) batch = (int64_t)((c->prob.t_end - cur.t) / cur.dt) + 1;
    batch = std::max<int64_t>(1, std::min<int64_t>(batch, std::min<int64_t>(256, max_steps - done)));
    for (int64_t k = 0; k < batch; ++k) IPM_CK(c, cudaGraphLaunch(c->step_exec, c->stream));
    done += batch;
    st = ipm_sync_stats(c, &cur);
    if (st != IPM_OK) return st;
    if (cur.failed_cells) break;
  }
  if (s) *s = cur;
  return IPM_OK;
}

}  // extern "C"
