// noalloc.cu -- ipm_dual_solve_noalloc: the per-cell Newton dual solve on caller-owned device
// buffers, with every piece of scratch memory taken from one fixed, file-scope device array.
//
// Why: some callers cannot allocate device memory themselves. Typical cases are a host
// application whose device memory is fully owned by another allocator (a framework's caching
// pool that reserves the device, or a pre-sized memory budget handed to a plugin), and
// timing-critical loops that must not pay cudaMalloc's implicit synchronisation. For them this
// entry point allocates nothing: the caller passes inputs and outputs, and the scratch (basis and
// quadrature tables, the work-queue counter and step scalars, the cell list and, for large N*m,
// the per-CTA Hessian workspace) lives in g_noalloc_scratch below.
//
// The scratch array is IPM_NOALLOC_SCRATCH_BYTES (8 MiB) and every GPU that loads the library
// holds it until the process exits. All calls share it and it keeps the last call's contents;
// the counters that must start at zero are cleared at the start of every call. Calls whose work
// overlaps on the GPU (different streams, or different host threads) race on the scratch and must
// not be issued concurrently. Every call looks up the array's device address on the current device
// with cudaGetSymbolAddress (cheap next to the table upload), so the address is never stale, also
// after a cudaDeviceReset; the first call on a device also loads the library's kernels there, so it
// should come before any stream capture.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "ipm_host.h"

static __device__ __align__(256) unsigned char g_noalloc_scratch[IPM_NOALLOC_SCRATCH_BYTES];

namespace {

ipm_status noalloc_fail(ipm_status s, const std::string& msg) {
  ipm::set_global_error(msg);
  return s;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

using namespace ipm;

extern "C" ipm_status ipm_dual_solve_noalloc(int problem_kind, double gamma, const ipm_basis* basis,
                                             const ipm_quadrature* quad, const ipm_entropy* entropy,
                                             const ipm_options* options, int n_cells, const double* d_uhat,
                                             double* d_lam, double* d_nodal, int* d_iters, int* d_status,
                                             void* stream, ipm_stats* stats) {
  if (!basis || !quad || !entropy || !d_uhat || !d_lam || !d_nodal || !d_iters || !d_status)
    return noalloc_fail(IPM_EINVAL, "ipm_dual_solve_noalloc: NULL argument");
  if (n_cells < 1 || n_cells > IPM_NOALLOC_MAX_CELLS)
    return noalloc_fail(IPM_EINVAL, "ipm_dual_solve_noalloc: n_cells must be in 1..IPM_NOALLOC_MAX_CELLS");
  if (basis->p < 1 || basis->p > 3 || basis->total_degree < 0 || quad->n_per_dim < 1)
    return noalloc_fail(IPM_EINVAL, "ipm_dual_solve_noalloc: basis needs 1 <= p <= 3, M >= 0, n_per_dim >= 1");
  if (quad->kind != IPM_QUAD_GAUSS)
    return noalloc_fail(IPM_EINVAL, "ipm_dual_solve_noalloc: tensor Gauss rules only");
  int m, phys;
  if (problem_kind == IPM_BURGERS_1D) {
    m = 1;
    phys = PHYS_BURGERS;
  } else if (problem_kind == IPM_EULER_1D) {
    m = 3;
    phys = PHYS_EULER1D;
  } else {
    return noalloc_fail(IPM_EINVAL, "ipm_dual_solve_noalloc: problem kind must be Burgers 1-D or Euler 1-D");
  }
  int entk;
  if (entropy->kind == IPM_ENTROPY_QUADRATIC) entk = ENT_QUADRATIC;
  else if (entropy->kind == IPM_ENTROPY_BOUNDED_BARRIER) entk = ENT_BARRIER;
  else if (entropy->kind == IPM_ENTROPY_EULER) entk = ENT_EULER;
  else return noalloc_fail(IPM_EINVAL, "ipm_dual_solve_noalloc: unknown entropy kind");
  if (!(entk == ENT_QUADRATIC || (entk == ENT_BARRIER && phys == PHYS_BURGERS) ||
        (entk == ENT_EULER && phys != PHYS_BURGERS)))
    return noalloc_fail(IPM_EINVAL, "ipm_dual_solve_noalloc: entropy does not match the problem");
  ipm_options opt;
  if (options) opt = *options;
  else ipm_default_options(&opt);
  if (opt.precision != IPM_PREC_FP64) return noalloc_fail(IPM_EINVAL, "ipm_dual_solve_noalloc: FP64 only");

  HostTables tab;
  build_tables(basis->p, basis->total_degree, quad->n_per_dim, tab);
  const int N = tab.N, Q = tab.Q, NM = N * m;
  if (N > 65535) return noalloc_fail(IPM_EINVAL, "ipm_dual_solve_noalloc: too many moments");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(IPM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  // The array's name is a host-side stand-in in host code; the kernels get its device address on the
  // current device, looked up on every call.
  void* base = nullptr;
  e = cudaGetSymbolAddress(&base, g_noalloc_scratch);
  if (e != cudaSuccess) return noalloc_fail(IPM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));

  int smem_optin = 0, n_sm = 0;
  e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return noalloc_fail(IPM_ECUDA, std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));
  const NewtonSmem sm_full = newton_smem(N, m, Q, true, nullptr);
  const NewtonSmem sm_lean = newton_smem(N, m, Q, false, nullptr);
  if (sm_lean.bytes > (size_t)smem_optin)
    return noalloc_fail(IPM_EINVAL, "ipm_dual_solve_noalloc: N*m and Q too large for one CTA");
  const bool h_in_smem = sm_full.bytes <= (size_t)smem_optin;
  const NewtonSmem sm = h_in_smem ? sm_full : sm_lean;
  const size_t smem = sm.bytes;
  int bps = 0;
  e = prepare_newton(entk, phys, m, smem, h_in_smem, 0, &bps);
  if (e != cudaSuccess || bps < 1) return noalloc_fail(IPM_ECUDA, std::string("kernel set-up: ") + cudaGetErrorString(e));

  // carve the scratch: scalars | Phi | PhiT | w | nodes | pairs | cell list | Hessian slots
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align256(off + bytes);
    return at;
  };
  const size_t o_sc = take(sizeof(StepScalars));
  const size_t o_phi = take(tab.Phi.size() * sizeof(double));
  const size_t o_phit = take(tab.PhiT.size() * sizeof(double));
  const size_t o_w = take(tab.w.size() * sizeof(double));
  const size_t o_nodes = take(tab.nodes.size() * sizeof(double));
  const size_t o_pairs = take(tab.pairs.size() * sizeof(uint32_t));
  const size_t o_cells = take((size_t)n_cells * sizeof(int));
  if (off > IPM_NOALLOC_SCRATCH_BYTES)
    return noalloc_fail(IPM_EINVAL, "ipm_dual_solve_noalloc: tables and cell list exceed the scratch size");
  int grid = std::max(1, std::min(n_cells, bps * n_sm));
  const size_t hslot = h_in_smem ? 0 : packed_aug_count(NM) * sizeof(double);
  size_t o_h = off;
  if (!h_in_smem) {
    const size_t room = IPM_NOALLOC_SCRATCH_BYTES - off;
    const int fit = (int)(room / hslot);
    if (fit < 1) return noalloc_fail(IPM_EINVAL, "ipm_dual_solve_noalloc: one Hessian workspace slot exceeds the scratch size");
    grid = std::min(grid, fit);
  }
  unsigned char* b = static_cast<unsigned char*>(base);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<int> cells(n_cells);
  for (int k = 0; k < n_cells; ++k) cells[k] = k;

  // clear the scalars (queue counter, speed maximum) and upload this call's tables
  e = cudaMemsetAsync(b + o_sc, 0, sizeof(StepScalars), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_phi, tab.Phi.data(), tab.Phi.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_phit, tab.PhiT.data(), tab.PhiT.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_w, tab.w.data(), tab.w.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_nodes, tab.nodes.data(), tab.nodes.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_pairs, tab.pairs.data(), tab.pairs.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_cells, cells.data(), cells.size() * sizeof(int), cudaMemcpyHostToDevice, s);
  // the host vectors above must outlive the copies from pageable memory
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return noalloc_fail(IPM_ECUDA, std::string("scratch upload: ") + cudaGetErrorString(e));

  NewtonArgs a;
  std::memset(&a, 0, sizeof(a));
  a.tab.Phi = reinterpret_cast<const double*>(b + o_phi);
  a.tab.PhiT = reinterpret_cast<const double*>(b + o_phit);
  a.tab.w = reinterpret_cast<const double*>(b + o_w);
  a.tab.nodes = reinterpret_cast<const double*>(b + o_nodes);
  a.tab.pairs = reinterpret_cast<const uint32_t*>(b + o_pairs);
  a.tab.N = N;
  a.tab.Q = Q;
  a.tab.p = tab.p;
  a.ent.u_minus = entropy->u_minus;
  a.ent.u_plus = entropy->u_plus;
  a.ent.gamma = gamma;
  a.uhat = const_cast<double*>(d_uhat);
  a.lam = d_lam;
  a.unode = d_nodal;
  a.iters = d_iters;
  a.status = d_status;
  a.hwork = h_in_smem ? nullptr : reinterpret_cast<double*>(b + o_h);
  a.hwork_stride = h_in_smem ? 0 : hslot / sizeof(double);
  a.sc = reinterpret_cast<StepScalars*>(b + o_sc);
  a.cell_list = reinterpret_cast<const int*>(b + o_cells);
  a.n_work = n_cells;
  a.nx = n_cells;
  a.gy = 0;
  a.one_step = 0;
  a.tau = opt.newton_tol;
  a.armijo_c = opt.armijo_c;
  a.slack_rel = opt.slack_rel;
  a.max_newton = opt.max_newton;
  a.max_halvings = opt.max_halvings;
  a.track_speed = 0;
  a.h_dump = nullptr;
  a.off_h = sm.off_h;
  e = launch_newton_phys(entk, phys, m, a, grid, smem, h_in_smem, 0, s);
  if (e == cudaSuccess) e = launch_finalize(a.sc, d_iters, d_status, nullptr, n_cells, 0, n_cells, 0, s);
  if (e != cudaSuccess) return noalloc_fail(IPM_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  if (stats) {
    StepScalars h;
    e = cudaMemcpyAsync(&h, a.sc, sizeof(StepScalars), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return noalloc_fail(IPM_ECUDA, std::string("stats: ") + cudaGetErrorString(e));
    std::memset(stats, 0, sizeof(*stats));
    stats->newton_iters = h.newton_iters;
    stats->max_iters = h.max_iters;
    stats->failed_cells = h.failed_cells;
    stats->first_failed_cell = h.first_failed_cell;
    stats->first_status = h.first_status;
  }
  return IPM_OK;
}
