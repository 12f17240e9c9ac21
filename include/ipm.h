/*
 * ipm.h -- C ABI of the GB300 Intrusive Polynomial Moment (IPM) library.
 *
 * The library runs the hot path of the IPM method for hyperbolic conservation laws with
 * uncertain initial data (Kusch, Wolters, Frank, "Intrusive acceleration strategies for
 * Uncertainty Quantification for hyperbolic systems of conservation laws", arXiv:1912.09238):
 *
 *   - the per-cell dual problem lambda_hat(u_hat) = argmin L(lambda; u_hat)         (Sec. 2, Eq. dualProblem;
 *     Sec. 3.1, Eq. L), solved by the Newton map d (Eq. dualIterationFunction) with an Armijo
 *     line search, stopped by Eq. tauCrit;
 *   - the kinetic-flux moment update c (Eq. momentIterationFunction, quadrature form
 *     Eq. momentUpQuadrature) with a Lax-Friedrichs flux (App. A);
 *   - Algorithm 1 (IPM time step) and Algorithm 2 (One-Shot IPM pseudo-time step).
 *
 * Conventions shared by every call
 *   Moments and duals cross the ABI as float64 arrays laid out [cell][moment][variable]
 *   (row-major), i.e. element (c, i, a) sits at c*N*m + i*m + a. "cell" runs over ALL cells
 *   including the ghost layer: 1-D meshes have nx+2 cells (ghost 0, interior 1..nx, ghost
 *   nx+1). "moment" i follows the graded total-degree order of the multi-indices: ascending
 *   total degree, and within one degree descending lexicographic order of (i_1..i_p)
 *   (Sec. 2, Eq. numberBasisFcts gives their number N = C(M+p, p)). "variable" a runs over the m
 *   conserved quantities (Burgers: u; 1-D Euler: rho, rho v, E; 2-D Euler: rho, rho v1,
 *   rho v2, E).
 *
 *   Ownership: ipm_init allocates all device state and keeps it resident until ipm_destroy.
 *   Host pointers passed in are only read (or written) during the call. Device-pointer calls
 *   (suffix _device) borrow the caller's buffer for the duration of the call and order their
 *   work on the context's stream.
 *
 *   Errors: every call returns an ipm_status; nothing throws or exits across the ABI. The
 *   message of the last failure is returned by ipm_last_error(ctx) (ctx may be NULL for a
 *   failure inside ipm_init). Per-cell solver failures do not fail the call: they are counted
 *   in ipm_stats, and the first failing cell and its status are reported there.
 *
 *   Threading: a context is not thread-safe; use one context per host thread. All GPU work of a
 *   context is ordered on its stream (ipm_set_stream).
 */
#ifndef IPM_H
#define IPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IPM_OK = 0,
  IPM_EINVAL = 1,       /* bad argument or unsupported combination */
  IPM_ENOMEM = 2,       /* device or host allocation failed */
  IPM_ENOCONV = 3,      /* Newton iteration cap reached (per-cell status) */
  IPM_ENOTSPD = 4,      /* Hessian not positive definite in the Cholesky factorisation (per-cell) */
  IPM_EINFEASIBLE = 5,  /* dual state outside the domain of u_s, e.g. Lambda_E >= 0 (per-cell) */
  IPM_ELINESEARCH = 6,  /* Armijo backtracking exhausted its halvings (per-cell) */
  IPM_ENONFINITE = 7,   /* NaN/Inf gradient (per-cell) */
  IPM_EAGAIN = 8,       /* serving: result not ready yet */
  IPM_ECUDA = 9,        /* a CUDA runtime call failed; see ipm_last_error */
  IPM_ETIMEOUT = 10     /* a bounded wait ran out */
} ipm_status;

typedef enum { IPM_BURGERS_1D = 0, IPM_EULER_1D = 1, IPM_EULER_2D = 2 } ipm_problem_kind;

/* Boundary handling of the ghost layer (Algorithm 1 keeps ghost cells j = 0, nx+1). */
typedef enum {
  IPM_BC_OUTFLOW = 0,    /* ghost copies its interior neighbour (moments and duals) */
  IPM_BC_PERIODIC = 1,   /* ghost copies the opposite interior cell */
  IPM_BC_DIRICHLET = 2,  /* ghost keeps its initial state; its duals are converged once at init */
  IPM_BC_SLIP_WALL = 3   /* 2-D only: wall; the outside state is the cell's own with the momentum
                            reflected about the face (Sec. 7 reflecting walls) */
} ipm_bc;

/* 2-D meshes (structured quadrilaterals, nx x ny interior cells, one ghost layer). */
typedef enum {
  IPM_MESH_CARTESIAN = 0,  /* [x_lo, x_hi] x [y_lo, y_hi], uniform */
  IPM_MESH_RAMP = 1        /* x in [x_lo, x_hi]; lower wall y_b(x) = y_lo, rising at ramp_deg degrees from
                              x = ramp_x0; top y_hi; rows mapped linearly y = y_b + (y_hi - y_b) eta */
} ipm_mesh_kind;

typedef enum {
  IPM_IC_RIEMANN = 0,    /* one jump at x0(xi); left/right primitive states affine in xi. In 2-D the jump
                            is at the fixed x = ic_x0, uniform in y, primitives (rho, v1, v2, p) */
  IPM_IC_FREESTREAM = 1, /* 2-D: uniform state; ic_param = (rho, p, Mach, flow angle in degrees), Mach and
                            angle affine in xi (ic_dparam[2], ic_dparam[3]); v = Mach c (cos, sin) */
  IPM_IC_SHEAR = 2       /* 2-D: band |y - (y_lo+y_hi)/2| < w(xi) with ic_left = (rho, v1, -, p) inside and
                            ic_right = (rho, v1, -, -) outside (pressure ic_left[3] everywhere), transverse
                            velocity v2 = A(xi) sin(k (x + phase(xi))); ic_param = (A, phase, w, k) with
                            ic_dparam rows their xi-derivatives. The band is averaged exactly over each cell's
                            y-extent; v2 is taken at the cell centre's x */
} ipm_ic_kind;

typedef enum {
  IPM_ENTROPY_QUADRATIC = 0,        /* s(u) = |u|^2/2: IPM = stochastic Galerkin (Sec. 1, Sec. 3.1) */
  IPM_ENTROPY_BOUNDED_BARRIER = 1,  /* s(u) = (u-u_-)ln(u-u_-) + (u_+-u)ln(u_+-u), scalar problems */
  IPM_ENTROPY_EULER = 2             /* s(u) = -rho ln(rho^-gamma (E - |m|^2/(2 rho)))  (App. B) */
} ipm_entropy_kind;

typedef enum {
  IPM_PREC_FP64 = 0,   /* every operation in float64 */
  IPM_PREC_MIXED = 1,  /* Hessian contraction on the tensor cores (BF16 split products, FP32
                          accumulate); gradient, Cholesky, Newton step and update in float64 */
  IPM_PREC_MIXED_F32_FACTOR = 2  /* as IPM_PREC_MIXED, but the Cholesky factorisation and the
                          triangular solves of the Newton direction run in FP32 on the CUDA cores
                          (the split-BF16 Hessian is accurate to ~3e-5 already, the FP32 factor to
                          ~n * 6e-8 relative); a cell whose FP32 factorisation meets a non-positive
                          pivot is refactorised in FP64. Gradient, stopping test (Eq. tauCrit), line
                          search and update stay float64, so the converged duals meet the same FP64
                          criterion. CTA-per-cell kernel only; not with frozen Hessians. */
} ipm_precision;

/* Problem description. Primitive states are (u) for Burgers and (rho, v_1[, v_2], p) for Euler;
 * every parameter X of the initial data is X + sum_d dX[d] * xi_d with xi_d ~ U[-1, 1].
 * 2-D Euler (Sec. 7): cells [j][i] with ghosts, cell index (j+1)*(nx+2) + (i+1) for interior i < nx,
 * j < ny; the moment update sums local Lax-Friedrichs (Rusanov) fluxes over the four faces of each
 * cell (face normals and lengths of the mapped mesh), dt = cfl * h / max speed with h the smallest
 * cell area over its longest face. */
typedef struct {
  int kind;                 /* ipm_problem_kind */
  int nx, ny;               /* interior cells (ny = 1 for 1-D problems) */
  double x_lo, x_hi;        /* 1-D domain */
  int bc_left, bc_right;    /* ipm_bc of the two 1-D ends */
  double cfl;               /* dt = cfl * dx / max speed over all cells and nodes */
  double t_end;             /* final time of ipm_run and clip of the last step; 0 = no clip */
  double gamma;             /* heat capacity ratio (Euler) */
  int ic_kind;              /* ipm_ic_kind */
  double ic_x0, ic_dx0[3];
  double ic_left[4], ic_dleft[4][3];
  double ic_right[4], ic_dright[4][3];
  /* 2-D problems (kind IPM_EULER_2D); ignored in 1-D */
  double y_lo, y_hi;        /* y range (IPM_MESH_RAMP: wall baseline and top) */
  int bc_bottom, bc_top;    /* ipm_bc of the lower and upper sides (bc_left / bc_right: x sides) */
  int mesh_kind;            /* ipm_mesh_kind */
  double ramp_x0, ramp_deg; /* IPM_MESH_RAMP geometry */
  double ic_param[4], ic_dparam[4][3];
} ipm_problem;

typedef struct {
  int p;                    /* number of uncertain dimensions, 1..3 */
  int total_degree;         /* M: moments N = C(M+p, p) */
} ipm_basis;

typedef enum {
  IPM_QUAD_GAUSS = 0,       /* tensor Gauss-Legendre rule with n_per_dim^p nodes (every level shares it) */
  IPM_QUAD_CC_NESTED = 1    /* nested tensor Clenshaw-Curtis rules, one per refinement level (Sec. 5: nested
                               quadrature per level; Sec. 7: Clenshaw-Curtis levels with 2^k + 1 points) */
} ipm_quad_kind;

typedef struct {
  int n_per_dim;            /* IPM_QUAD_GAUSS: nodes per dimension */
  int kind;                 /* ipm_quad_kind; 0 (a zero-initialised struct) is the Gauss rule */
  int cc_level[8];          /* IPM_QUAD_CC_NESTED: Clenshaw-Curtis level k_l of refinement level l (adaptive
                               contexts, l = 0 .. levels-1; fixed degree: cc_level[0]); the 1-D rule of level
                               k has 2^k + 1 points (k = 0: the midpoint); k_l must not decrease with l, must
                               give 2^k_l + 1 >= M_l + 1 points per dimension and be at most 6. All zero: the
                               smallest k >= 1 with 2^k + 1 >= M_l + 2. The finest level's rule is the node
                               set of the context: nodal arrays hold (2^k_max + 1)^p nodes, ordered so that
                               every coarser level's nodes come first. A cell of level l solves its dual
                               problem with the level-l rule (Eq. dualIterationFunctionAd); its moment update
                               integrates with the rule of its new level, with every stencil cell's ansatz
                               evaluated at those nodes (Eq. adaptiveFVUpdate); the time step takes each
                               cell's wave speed at the nodes of its new level. */
} ipm_quadrature;

typedef struct {
  int kind;                 /* ipm_entropy_kind */
  double u_minus, u_plus;   /* bounded barrier bounds */
} ipm_entropy;

typedef struct {
  int precision;            /* ipm_precision */
  double newton_tol;        /* tau of Eq. tauCrit (absolute; sum over moments of 2-norms) */
  int max_newton;           /* Newton iteration cap per cell and solve */
  double armijo_c;          /* sufficient-decrease constant */
  int max_halvings;         /* Armijo backtracking cap */
  double slack_rel;         /* rounding allowance of the Armijo test, relative to the terms of L */
  /* Adaptive IPM (Sec. 5, Algorithm 3; 2-D problems): 0 = off; else every cell carries a total degree
   * between adapt_min_degree and basis.total_degree (at most 8 levels), chosen each step by the
   * smoothness indicator S (Eq. errorIndicator) of its density moments: kept for S in
   * [min(delta_lo, delta_hi), max(...)], lowered one degree below, raised one above; the moments and
   * duals beyond a cell's degree are zero (graded ordering: a lower degree is a prefix). */
  int adapt_min_degree;
  double delta_lo, delta_hi;
  /* Frozen Hessians (the paper's outlook, Sec. 8: quasi-Newton / frozen Hessians): 0 = Newton (the
   * paper's method); 1 = after the first update of a solve, keep using the last Cholesky factor while the
   * previous step was a full step (alpha = 1) and reduced the stopping criterion by at least reuse_ratio,
   * else refactorise; 2 = like 1, and the newest factor of every cell is kept between solves (device
   * memory n_cells * (N*m(N*m+1)/2 + N*m) doubles, refused with IPM_EINVAL above a quarter of the free
   * memory) and used for the first update of the next solve. The converged duals meet the same FP64
   * criterion (Eq. tauCrit) as Newton's. Runs on the CTA-per-cell Newton kernel. */
  int hessian_reuse;
  double reuse_ratio;
  /* Newton kernel: 0 = autotune (time each applicable variant on the initial state at ipm_init and
   * keep the fastest; the decision is remembered for the process, per problem shape (kind, entropy,
   * N, m, Q, precision, power-of-two bucket of the interior cell count), so equal shapes always run
   * the same variant), 1 = one CTA per cell, 2 = one warp per cell (cells with N*m <= 64, fixed degree).
   * Adaptive meshes solve the cells of their lowest levels with N*m <= 64 one warp per cell (nodes in
   * chunks of 32) and the others one CTA per cell; 1 keeps every cell on the CTA kernel. */
  int newton_kernel;
  /* Convergence checks from moment images (fixed-degree meshes on the CTA-per-cell kernel; adaptive
   * meshes with one quadrature rule for every level, on both of their kernels): 1 (default) = every
   * cell keeps S = sum_k w_k u(Lambda(xi_k)) phi(xi_k) of the duals its last successful solve ended at,
   * with those duals and its level; a solve that starts from the same duals (bit for bit) at the same
   * level takes its first gradient as S - u_hat, which is the gradient of Eq. gradient with the same
   * arithmetic, and a cell that meets Eq. tauCrit there skips the reconstruction and the closures.
   * Results are identical to 0 (always evaluate); device memory 2 n_cells N m doubles. */
  int check_cache;
  /* Cholesky factorisation of the Newton step (row (c), Sec. 3.1), CTA-per-cell kernel: 1 = blocked
   * right-looking factorisation with FP64 FMAs on the CUDA cores; 2 = split factorisation: the same
   * factorisation with 16-column panels factorised in FP64 and every trailing update L21 L21^T computed
   * exactly on the tensor cores from base-256 digit slices of L21 (seven BF16 digits per entry, one
   * scale per row, FP32 accumulators that hold every diagonal of digit products exactly), combined in
   * 64-bit integers and applied with one FP64 FMA: FP64-level accuracy; 0 (default) = 2 on
   * IPM_PREC_MIXED for N*m >= 128, else 1. Not with IPM_PREC_MIXED_F32_FACTOR (IPM_EINVAL). */
  int factorization;
} ipm_options;

/* Sizes of a context's arrays. */
typedef struct {
  int N;                    /* moments per variable */
  int m;                    /* conserved variables */
  int Q;                    /* quadrature nodes */
  int p;                    /* uncertain dimensions */
  int n_cells;              /* all cells including ghosts */
  int n_interior;           /* interior cells */
} ipm_dims;

/* Counters of the last solve or step. */
typedef struct {
  int64_t newton_iters;     /* Newton updates summed over cells */
  int32_t max_iters;        /* largest per-cell count */
  int32_t failed_cells;     /* cells whose per-cell status is not IPM_OK */
  int32_t first_failed_cell;/* lowest failing cell index, -1 if none */
  int32_t first_status;     /* its ipm_status */
  double dt;                /* time step taken (ipm_step / ipm_oneshot_step) */
  double t;                 /* time after the call */
  double residual;          /* steady residual of the last step (Eq. residualSteady, first variable) */
  int64_t steps;            /* steps taken since ipm_init */
  int32_t tc_timeouts;      /* mixed path: bounded tensor-core / bulk-copy waits that ran out (0 normally;
                               the affected cells report IPM_ETIMEOUT). If a CTA then cannot drain its
                               outstanding tensor-core work either, it keeps its tensor memory, the
                               stats call returns IPM_ETIMEOUT and every later launching call on the
                               context returns IPM_ETIMEOUT without launching: destroy the context. */
  int64_t factorizations;   /* Cholesky factorisations of the last solve (equals newton_iters without
                               frozen Hessians) */
  int32_t fp32_fallbacks;   /* IPM_PREC_MIXED_F32_FACTOR: FP32 factorisations redone in FP64 (cumulative) */
  int64_t cached_checks;    /* cells of the last solve whose convergence check came from their moment
                               image (ipm_options.check_cache) */
  int64_t hessian_ns;       /* mixed paths, CTA-per-cell kernel: summed duration of the last solve's
                               tensor-core Hessian assemblies (row (b) of Sec. 3.1), each timed on the
                               device from its start to its last barrier; 0 on the FP64 path */
  int64_t hessian_count;    /* ... the number of assemblies that sum covers */
} ipm_stats;

typedef struct ipm_ctx ipm_ctx;

/* Fill *opt with the defaults: FP64, tau = 1e-10, 100 iterations, c = 1e-4, 30 halvings,
 * slack 1e-12, no adaptivity (thresholds 2e-5 and 2e-4 preset). */
void ipm_default_options(ipm_options* opt);

/* Create a context on the current CUDA device: build the basis and quadrature tables, allocate
 * the resident state, project the initial data (Algorithm 1, first loop) and set the initial
 * duals to the projection of the nodal entropy variables; Dirichlet ghosts are solved to
 * convergence. Returns IPM_EINVAL for unsupported sizes (N*m above the per-CTA limit of the
 * chosen precision), IPM_ENOMEM / IPM_ECUDA on device failures. */
ipm_status ipm_init(const ipm_problem* problem, const ipm_basis* basis, const ipm_quadrature* quad,
                    const ipm_entropy* entropy, const ipm_options* options, ipm_ctx** out);

/* Release all device state of ctx. NULL is accepted. */
void ipm_destroy(ipm_ctx* ctx);

/* Message of the last failing call on ctx (or of the last failing ipm_init when ctx is NULL). */
const char* ipm_last_error(const ipm_ctx* ctx);

ipm_status ipm_get_dims(const ipm_ctx* ctx, ipm_dims* out);

/* Order all later work of ctx on the given cudaStream_t, used verbatim: NULL is the CUDA legacy
 * default stream (the stream PyTorch reports as 0). Until the first call the context uses a
 * non-blocking stream of its own. Waits for the work already queued on the previous stream. The
 * context's device memory comes from a stream-ordered pool and is released on its current stream by
 * ipm_destroy, so a stream given here must stay valid until the context is destroyed (or another
 * stream is set). */
ipm_status ipm_set_stream(ipm_ctx* ctx, void* cuda_stream);

/* Copy moments / duals in or out; count must equal n_cells*N*m doubles. Synchronous. */
ipm_status ipm_set_moments(ipm_ctx* ctx, const double* host, size_t count);
ipm_status ipm_get_moments(ipm_ctx* ctx, double* host, size_t count);
ipm_status ipm_set_duals(ipm_ctx* ctx, const double* host, size_t count);
ipm_status ipm_get_duals(ipm_ctx* ctx, double* host, size_t count);
/* Clock of a context: simulated (or pseudo-) time, last time step, steps taken, and the level cap of
 * Algorithm 4 (adaptive contexts; levels - 1 without retardation). */
typedef struct {
  double t;
  double dt;
  int64_t steps;
  int32_t level_cap;
} ipm_clock;

/* Checkpoint / resume: the whole state of a context in one call with one synchronisation -- moments
 * and duals ([cell][moment][variable] each, count = n_cells*N*m doubles per array), the refinement
 * level of every cell (adaptive contexts: n_cells ints; NULL to skip, and ignored on fixed-degree
 * contexts) and the clock (NULL to skip). A context restored from a checkpoint of a context of the
 * same problem continues bit for bit as the original would (kept Cholesky factors of hessian_reuse 2
 * are not part of the state: a restored context refactorises, so its iterates differ within the
 * stopping tolerance). Also the way to stream a step's state in and out. */
ipm_status ipm_set_state(ipm_ctx* ctx, const double* moments, const double* duals, const int* levels,
                         const ipm_clock* clock, size_t count);
ipm_status ipm_get_state(ipm_ctx* ctx, double* moments, double* duals, int* levels, ipm_clock* clock,
                         size_t count);
/* Nodal states u_s(lambda_j^T phi(xi_k)) at the current duals, laid out [cell][variable][node]
 * (count = n_cells*m*Q). Valid after ipm_dual_solve / ipm_step / ipm_oneshot_step. */
ipm_status ipm_get_nodal_states(ipm_ctx* ctx, double* host, size_t count);

/* Adaptive contexts, Algorithm 4 (refinement retardation, Sec. 5): from now on no interior cell may go
 * above level max_level (index from adapt_min_degree); cells above it are lowered at once (moments and
 * duals beyond it set to zero). Dirichlet ghosts keep their initial levels. */
ipm_status ipm_set_max_level(ipm_ctx* ctx, int max_level);

/* Algorithm 4 (adaptive One-Shot IPM with refinement retardation) on an adaptive context: stage l
 * allows levels up to max_levels[l]; One-Shot pseudo-time steps (ipm_oneshot_step) run until the steady
 * residual (Eq. residualSteady) falls below tolerances[l], then the next stage begins; in the last
 * stage the run stops at residual tol. At most max_steps steps; *stats holds the last step's counters
 * and stats->steps the steps taken so far. Synchronous (reads the residual after every step). */
ipm_status ipm_oneshot_retarded(ipm_ctx* ctx, const int* max_levels, const double* tolerances, int n_stages,
                                double tol, int64_t max_steps, ipm_stats* stats);

/* The Newton kernel variant in use (1 = CTA per cell, 2 = warp per cell) and the times of one
 * Newton solve on the initial state measured by the autotuner (0 for a variant not timed). */
ipm_status ipm_get_tuning(const ipm_ctx* ctx, int* kernel, float* ms_cta, float* ms_warp);

/* Adaptive contexts: the refinement level (index from adapt_min_degree) of every cell, count = n_cells. */
ipm_status ipm_get_levels(ipm_ctx* ctx, int* host, size_t count);

/* Device-pointer variants: buffers live on the context's device, same layout and count;
 * asynchronous on the context's stream. */
ipm_status ipm_set_moments_device(ipm_ctx* ctx, const double* dev, size_t count);
ipm_status ipm_get_moments_device(ipm_ctx* ctx, double* dev, size_t count);

/* Newton solve of the dual problem in every interior cell (Eq. dualIteration1 until Eq. tauCrit),
 * warm-started at the current duals; the nodal states of the result are kept for the next
 * update. Synchronous when stats != NULL. */
ipm_status ipm_dual_solve(ipm_ctx* ctx, ipm_stats* stats);

/* The Hessian H((i,a),(j,b)) = sum_k w_k [grad u_s]_ab(Lambda_k) phi_i(xi_k) phi_j(xi_k) of the dual
 * cost (Sec. 3.1, the Jacobian of the Newton map of Eq. dualIterationFunction) at the current duals of
 * every interior cell, assembled exactly as the Newton kernel assembles it in the context's
 * precision (IPM_PREC_MIXED: split-BF16 tensor-core products with FP32 accumulation, widened to
 * float64). Output: packed lower triangles, host array [interior cell][r(r+1)/2 + c] for r >= c with
 * flat index r = i*m + a; count = n_interior * N*m*(N*m+1)/2. Does not change the state (the nodal
 * states are refreshed at the current duals). Allocates a temporary device buffer; synchronous. */
ipm_status ipm_assemble_hessian(ipm_ctx* ctx, double* host, size_t count);

/* The Cholesky factor L (H = L L^T, row (c) of Sec. 3.1, Eq. dualIterationFunction's linear solve) of
 * the Hessian that ipm_assemble_hessian returns at the current duals of every interior cell, computed
 * by the context's factorisation (ipm_options.factorization; IPM_PREC_MIXED_F32_FACTOR contexts report
 * their FP64 fallback factorisation). Same layout and count as ipm_assemble_hessian (packed lower
 * triangles, L's diagonal included); a cell whose Hessian is not numerically SPD leaves its slice
 * unspecified and is reported by the next ipm_sync_stats. Does not change the state. Allocates a
 * temporary device buffer; synchronous. */
ipm_status ipm_factor_hessian(ipm_ctx* ctx, double* host, size_t count);

/* Only the moment update c of every interior cell from the current duals (Eq. momentUpQuadrature)
 * with the given dt > 0 (dt is not computed and t is not advanced); then the boundary condition.
 * Requires a preceding ipm_dual_solve. */
ipm_status ipm_update(ipm_ctx* ctx, double dt);

/* One time step of Algorithm 1: dual solve in every cell, dt from the CFL rule on the new nodal
 * states (clipped to t_end), moment update, boundary condition. Runs as one captured CUDA graph.
 * Asynchronous when stats == NULL; otherwise waits and fills *stats. */
ipm_status ipm_step(ipm_ctx* ctx, ipm_stats* stats);

/* Steps of Algorithm 1 until t >= t_end (at most max_steps); fills *stats if not NULL. */
ipm_status ipm_run(ipm_ctx* ctx, int64_t max_steps, ipm_stats* stats);

/* One pseudo-time step of Algorithm 2 (One-Shot IPM): one damped Newton step per interior cell,
 * ghost duals from the boundary condition, moment update with the CFL dt, steady residual
 * (Eq. residualSteady on the zero-order moment of the first variable) into stats->residual. */
ipm_status ipm_oneshot_step(ipm_ctx* ctx, ipm_stats* stats);

/* Device time of the last ipm_step / ipm_oneshot_step, from CUDA events recorded inside its graph:
 * the Newton kernel (with its queue reset), the moment update, and the whole step. Waits for the
 * step to finish. Any output may be NULL. */
ipm_status ipm_step_timing(ipm_ctx* ctx, float* newton_ms, float* update_ms, float* total_ms);

/* Wait for the context's stream and fill *stats with the counters of the last step or solve. */
ipm_status ipm_sync_stats(ipm_ctx* ctx, ipm_stats* stats);

/* Scratch limits of ipm_dual_solve_noalloc: one static device array of this many bytes per GPU
 * that loads the library, and at most this many cells per call. */
#define IPM_NOALLOC_SCRATCH_BYTES (8u << 20)
#define IPM_NOALLOC_MAX_CELLS 262144

/* Dual solve that allocates nothing (the paper has no counterpart: this is a library-usage
 * variant of ipm_dual_solve). For callers that cannot allocate device memory themselves -- their
 * device memory is owned by another allocator (a framework's caching pool or a fixed budget handed
 * to a plugin), or they run timing-critical loops that must not pay cudaMalloc's implicit
 * synchronisation. Solves the dual problem (Newton until tau) in every one of n_cells cells of
 * caller-owned device buffers, on the given stream (NULL = legacy default stream):
 *   d_uhat   [n_cells][N][m] moments (in);  d_lam [n_cells][N][m] duals (in: warm start, out: result);
 *   d_nodal  [n_cells][m][Q] nodal states u_s at the result (out);
 *   d_iters, d_status [n_cells] Newton updates and ipm_status per cell (out).
 * All scratch (tables, counters, cell list, Hessian workspace) comes from one file-scope device
 * array of IPM_NOALLOC_SCRATCH_BYTES that every GPU loading the library keeps until exit; no
 * cudaMalloc, cudaFree or allocating library routine is called. Sizes beyond the scratch (or more
 * than IPM_NOALLOC_MAX_CELLS cells) return IPM_EINVAL with a message in ipm_last_error(NULL).
 * Calls share the array and it keeps the last call's contents (counters are cleared at the start
 * of each call); calls that overlap on the GPU race and must not be issued concurrently. Every call
 * looks up the array's device address on the current device (cudaGetSymbolAddress); the first call
 * on a device also loads the library's kernels there, so make that first call before any stream
 * capture. Each call uploads its tables from host memory and waits on the stream for that upload;
 * with stats != NULL it also waits for the solve and fills the counters. Unknown problem or entropy
 * kinds return IPM_EINVAL. FP64 precision, 1-D problem kinds only. */
ipm_status ipm_dual_solve_noalloc(int problem_kind, double gamma, const ipm_basis* basis,
                                  const ipm_quadrature* quad, const ipm_entropy* entropy,
                                  const ipm_options* options, int n_cells, const double* d_uhat,
                                  double* d_lam, double* d_nodal, int* d_iters, int* d_status,
                                  void* stream, ipm_stats* stats);

/* Device bytes ipm_init would allocate for this problem (state, tables, workspaces), without
 * allocating anything. Validates the arguments like ipm_init (IPM_EINVAL on the same errors). */
ipm_status ipm_footprint(const ipm_problem* problem, const ipm_basis* basis, const ipm_quadrature* quad,
                         const ipm_entropy* entropy, const ipm_options* options, size_t* bytes);

/* ------------------------------------------------------------------------------------------------
 * Serving: a continuous-batching request server for IPM runs (the paper has no serving layer; this
 * is the library's request API around Algorithm 1).
 *
 * A server owns one worker thread on the device that was current at ipm_server_create. Submitted
 * requests wait in arrival order until a slot and device memory are free (admission by the
 * ipm_footprint of each request against the memory cap); an admitted request gets a resident context
 * (its moments and duals stay on the device for its whole run) on a stream of its own, and the worker
 * keeps launching its time steps (one CUDA graph each) interleaved with every other active request,
 * so the kernels of different requests overlap on the GPU. A request finishes when it reaches its
 * t_end (or max_steps); its final moments are copied to the host and its slot and memory are freed
 * for the next waiting request. Each request's results are independent of what else runs: the same
 * request gives the same moments alone and in any mix.
 * ------------------------------------------------------------------------------------------------ */
typedef struct ipm_server ipm_server;

typedef struct {
  ipm_problem problem;
  ipm_basis basis;
  ipm_quadrature quad;
  ipm_entropy entropy;
  ipm_options options;
  int64_t max_steps;        /* at most this many Algorithm-1 steps (problem.t_end > 0: stop at t_end) */
} ipm_request;

typedef struct {
  int32_t status;           /* ipm_status of the run: IPM_OK, or the first per-cell failure */
  ipm_dims dims;
  ipm_stats stats;          /* counters after the last step (t, steps, Newton updates of the last step) */
  double submit_s;          /* server clock (seconds since ipm_server_create) at ipm_submit */
  double start_s;           /* ... when the request was admitted */
  double finish_s;          /* ... when its final moments were on the host */
  size_t footprint_bytes;   /* ipm_footprint of the request */
  char error[192];          /* message of the failing call when status is not IPM_OK, else empty */
} ipm_result;

/* Create a server. mem_cap_bytes: device memory the active requests may hold together (0 = 90% of
 * the free device memory now); max_active: concurrent resident requests (slots), >= 1. */
ipm_status ipm_server_create(size_t mem_cap_bytes, int max_active, ipm_server** out);

/* Queue a request (copied); *ticket identifies it. IPM_EINVAL for a request ipm_init would reject,
 * IPM_ENOMEM if its footprint alone exceeds the cap. Thread-safe. */
ipm_status ipm_submit(ipm_server* srv, const ipm_request* req, uint64_t* ticket);

/* IPM_EAGAIN while the request is waiting or running. Once it is done: fills *out, and when moments
 * is not NULL copies its final moments ([cell][moment][variable], count = n_cells*N*m) and releases
 * the ticket (later polls of it return IPM_EINVAL). Thread-safe. */
ipm_status ipm_poll(ipm_server* srv, uint64_t ticket, ipm_result* out, double* moments, size_t count);

/* Block until every submitted request is done (or timeout_s seconds have passed: IPM_ETIMEOUT). */
ipm_status ipm_server_drain(ipm_server* srv, double timeout_s);

/* Stop the worker: waiting requests are dropped, running ones finish first. NULL is accepted. */
void ipm_server_destroy(ipm_server* srv);

/* Host-only: the nested Clenshaw-Curtis tables of level kmax (IPM_QUAD_CC_NESTED): nodes Q*p doubles
 * (Q = (2^kmax + 1)^p, coarser levels first), level_weights (kmax+1)*Q doubles (row k: the level-k
 * weights of the first (2^k + 1)^p nodes, density folded in, zero beyond), phi Q*N doubles. Any output
 * may be NULL; IPM_EINVAL for p outside 1..3, kmax outside 0..6 or too small capacities. */
ipm_status ipm_tables_cc(int p, int total_degree, int kmax, int N_cap, int Q_cap, int* indices, double* nodes,
                         double* level_weights, double* phi, int* N_out, int* Q_out);

/* Host-only: the basis and quadrature tables the library uses (no GPU needed).
 * indices: N*p ints (graded order), nodes: Q*p doubles, weights: Q doubles (density folded in,
 * summing to 1), phi: Q*N doubles with phi[k*N + i] = phi_i(xi_k). Any output may be NULL.
 * Returns IPM_EINVAL if p is outside 1..3 or a size exceeds the given capacities (N_cap, Q_cap). */
ipm_status ipm_tables(int p, int total_degree, int n_per_dim, int N_cap, int Q_cap,
                      int* indices, double* nodes, double* weights, double* phi, int* N_out, int* Q_out);

/* ---- Stochastic Collocation (SC): the non-intrusive baseline (Sec. 2, the collocation paragraph;
 * Sec. 7, the IPM-versus-SC comparisons) -------------------------------------------------------------
 * Every node xi_k of the tensor Gauss rule of (basis, quad) runs the deterministic finite-volume
 * scheme of the IPM update, with the same numerical flux (global Lax-Friedrichs in 1-D, Rusanov on 2-D
 * meshes) and the same boundary handling, on its own state u(x, t, xi_k), starting from the exact
 * nodal cell averages of the initial data. Each node is a black box: its own time step
 * dt_k = cfl * h / max wave speed of node k (interior and Dirichlet ghosts; h = dx in 1-D), with the
 * 1-D viscosity dx / (2 dt_k) of that step, and its own step count. Unsteady problems (t_end > 0)
 * stop each node at t_end (last step clipped); steady problems (t_end == 0) iterate each node until
 * its residual sum_c A_c |rho_c^{n+1} - rho_c^n| (A_c = dx in 1-D) is below steady_tol. The moments
 * are u_hat_i = sum_k w_k u(xi_k) phi_i(xi_k) (layout [cell][moment][variable] as everywhere).
 * The library has no entropy or dual state here: SC needs neither. */
typedef struct ipm_sc ipm_sc;

typedef struct {
  int64_t steps;            /* lockstep steps launched since ipm_sc_init (finished nodes are carried through) */
  int64_t max_node_steps;   /* most steps any node has taken */
  int32_t active_nodes;     /* nodes still running */
  double t_min, t_max;      /* smallest and largest node time */
  double residual_max;      /* largest last steady residual over the nodes (0 before the first step) */
  double elapsed_ms;        /* device time of this call's launches (CUDA events on the object's stream) */
} ipm_sc_stats;

/* Allocate the nodal states (two buffers of cells * nodes * variables float64) and set the initial
 * data. steady_tol is used (and must be > 0) when problem->t_end == 0. IPM_EINVAL for a problem
 * ipm_init would reject; IPM_ENOMEM / IPM_ECUDA as ipm_init. */
ipm_status ipm_sc_init(const ipm_problem* problem, const ipm_basis* basis, const ipm_quadrature* quad,
                       double steady_tol, ipm_sc** out);

/* One step of every running node; stats may be NULL. */
ipm_status ipm_sc_step(ipm_sc* sc, ipm_sc_stats* stats);

/* Step until every node has finished or max_steps lockstep steps have been launched in total
 * (steps are launched in captured graphs of 16; a node that finishes inside a graph is carried
 * through unchanged). stats may be NULL. */
ipm_status ipm_sc_run(ipm_sc* sc, int64_t max_steps, ipm_sc_stats* stats);

/* Nodal states [cell][node][variable] (count = cells * nodes * variables, ghosts included). */
ipm_status ipm_sc_get_nodal(ipm_sc* sc, double* host, size_t count);

/* SC moments [cell][moment][variable] (count = cells * N * variables). */
ipm_status ipm_sc_get_moments(ipm_sc* sc, double* host, size_t count);

/* Per node (count = node count; any output may be NULL): steps taken, time reached, last residual. */
ipm_status ipm_sc_get_node_info(ipm_sc* sc, int64_t* steps, double* t, double* residual, size_t count);

ipm_status ipm_sc_get_dims(const ipm_sc* sc, int* n_cells, int* n_nodes, int* n_moments, int* n_vars);
const char* ipm_sc_last_error(const ipm_sc* sc);   /* NULL: the last failure without a handle */
void ipm_sc_destroy(ipm_sc* sc);                   /* NULL is accepted */

#ifdef __cplusplus
}
#endif

#endif /* IPM_H */
