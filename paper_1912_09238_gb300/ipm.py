"""Thin ctypes binding of libipm (include/ipm.h). Argument marshalling only: every step of the IPM
path runs in the library's CUDA kernels. There is no CPU fallback: if libipm.so is missing or no
CUDA device is present the calls raise."""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libipm.so")

IPM_OK = 0
STATUS_NAMES = {0: "IPM_OK", 1: "IPM_EINVAL", 2: "IPM_ENOMEM", 3: "IPM_ENOCONV", 4: "IPM_ENOTSPD",
                5: "IPM_EINFEASIBLE", 6: "IPM_ELINESEARCH", 7: "IPM_ENONFINITE", 8: "IPM_EAGAIN",
                9: "IPM_ECUDA", 10: "IPM_ETIMEOUT"}
PROBLEM = {"burgers1d": 0, "euler1d": 1, "euler2d": 2}
BC = {"outflow": 0, "periodic": 1, "dirichlet": 2, "slip": 3}
MESH = {"cartesian": 0, "ramp": 1}
IC = {"riemann": 0, "freestream": 1, "shear": 2}
ENTROPY = {"quadratic": 0, "barrier": 1, "euler": 2}
PRECISION = {"fp64": 0, "mixed": 1, "mixed_f32f": 2}


class ipm_problem(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x_lo", ctypes.c_double), ("x_hi", ctypes.c_double),
                ("bc_left", ctypes.c_int), ("bc_right", ctypes.c_int),
                ("cfl", ctypes.c_double), ("t_end", ctypes.c_double), ("gamma", ctypes.c_double),
                ("ic_kind", ctypes.c_int), ("ic_x0", ctypes.c_double), ("ic_dx0", ctypes.c_double * 3),
                ("ic_left", ctypes.c_double * 4), ("ic_dleft", (ctypes.c_double * 3) * 4),
                ("ic_right", ctypes.c_double * 4), ("ic_dright", (ctypes.c_double * 3) * 4),
                ("y_lo", ctypes.c_double), ("y_hi", ctypes.c_double), ("bc_bottom", ctypes.c_int),
                ("bc_top", ctypes.c_int), ("mesh_kind", ctypes.c_int), ("ramp_x0", ctypes.c_double),
                ("ramp_deg", ctypes.c_double), ("ic_param", ctypes.c_double * 4),
                ("ic_dparam", (ctypes.c_double * 3) * 4)]


class ipm_basis(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("total_degree", ctypes.c_int)]


class ipm_quadrature(ctypes.Structure):
    _fields_ = [("n_per_dim", ctypes.c_int), ("kind", ctypes.c_int), ("cc_level", ctypes.c_int * 8)]


def quadrature(n_per_dim=0, cc_levels=None):
    """ipm_quadrature: the tensor Gauss rule with n_per_dim nodes per dimension, or (cc_levels given)
    nested Clenshaw-Curtis rules, cc_levels[l] the level of refinement level l (() = the default rule)."""
    q = ipm_quadrature(n_per_dim=n_per_dim)
    if cc_levels is not None:
        q.kind = 1
        for l, k in enumerate(cc_levels):
            q.cc_level[l] = k
    return q


def _quad(n_per_dim):
    return n_per_dim if isinstance(n_per_dim, ipm_quadrature) else ipm_quadrature(n_per_dim=n_per_dim)


class ipm_entropy(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("u_minus", ctypes.c_double), ("u_plus", ctypes.c_double)]


class ipm_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("newton_tol", ctypes.c_double), ("max_newton", ctypes.c_int),
                ("armijo_c", ctypes.c_double), ("max_halvings", ctypes.c_int), ("slack_rel", ctypes.c_double),
                ("adapt_min_degree", ctypes.c_int), ("delta_lo", ctypes.c_double), ("delta_hi", ctypes.c_double),
                ("hessian_reuse", ctypes.c_int), ("reuse_ratio", ctypes.c_double), ("newton_kernel", ctypes.c_int),
                ("check_cache", ctypes.c_int), ("factorization", ctypes.c_int)]


class ipm_dims(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("m", ctypes.c_int), ("Q", ctypes.c_int), ("p", ctypes.c_int),
                ("n_cells", ctypes.c_int), ("n_interior", ctypes.c_int)]


class ipm_stats(ctypes.Structure):
    _fields_ = [("newton_iters", ctypes.c_int64), ("max_iters", ctypes.c_int32), ("failed_cells", ctypes.c_int32),
                ("first_failed_cell", ctypes.c_int32), ("first_status", ctypes.c_int32),
                ("dt", ctypes.c_double), ("t", ctypes.c_double), ("residual", ctypes.c_double),
                ("steps", ctypes.c_int64), ("tc_timeouts", ctypes.c_int32), ("factorizations", ctypes.c_int64),
                ("fp32_fallbacks", ctypes.c_int32), ("cached_checks", ctypes.c_int64),
                ("hessian_ns", ctypes.c_int64), ("hessian_count", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ipm_request(ctypes.Structure):
    _fields_ = [("problem", ipm_problem), ("basis", ipm_basis), ("quad", ipm_quadrature), ("entropy", ipm_entropy),
                ("options", ipm_options), ("max_steps", ctypes.c_int64)]


class ipm_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("dims", ipm_dims), ("stats", ipm_stats), ("submit_s", ctypes.c_double),
                ("start_s", ctypes.c_double), ("finish_s", ctypes.c_double), ("footprint_bytes", ctypes.c_size_t),
                ("error", ctypes.c_char * 192)]


class ipm_clock(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("dt", ctypes.c_double), ("steps", ctypes.c_int64), ("level_cap", ctypes.c_int32)]


class ipm_sc_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("max_node_steps", ctypes.c_int64), ("active_nodes", ctypes.c_int32),
                ("t_min", ctypes.c_double), ("t_max", ctypes.c_double), ("residual_max", ctypes.c_double),
                ("elapsed_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class IpmError(RuntimeError):
    def __init__(self, call, status, msg):
        super().__init__(f"{call} -> {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None
_P = ctypes.POINTER
_vp = ctypes.c_void_p
_dp = _P(ctypes.c_double)

# (name, restype, argtypes): every entry point declared in include/ipm.h
SIGNATURES = [
    ("ipm_default_options", None, [_P(ipm_options)]),
    ("ipm_init", ctypes.c_int, [_P(ipm_problem), _P(ipm_basis), _P(ipm_quadrature), _P(ipm_entropy),
                                _P(ipm_options), _P(_vp)]),
    ("ipm_destroy", None, [_vp]),
    ("ipm_last_error", ctypes.c_char_p, [_vp]),
    ("ipm_get_dims", ctypes.c_int, [_vp, _P(ipm_dims)]),
    ("ipm_set_stream", ctypes.c_int, [_vp, _vp]),
    ("ipm_set_moments", ctypes.c_int, [_vp, _dp, ctypes.c_size_t]),
    ("ipm_get_moments", ctypes.c_int, [_vp, _dp, ctypes.c_size_t]),
    ("ipm_set_duals", ctypes.c_int, [_vp, _dp, ctypes.c_size_t]),
    ("ipm_get_duals", ctypes.c_int, [_vp, _dp, ctypes.c_size_t]),
    ("ipm_get_nodal_states", ctypes.c_int, [_vp, _dp, ctypes.c_size_t]),
    ("ipm_set_state", ctypes.c_int, [_vp, _dp, _dp, _P(ctypes.c_int), _vp, ctypes.c_size_t]),
    ("ipm_get_state", ctypes.c_int, [_vp, _dp, _dp, _P(ctypes.c_int), _vp, ctypes.c_size_t]),
    ("ipm_get_levels", ctypes.c_int, [_vp, _P(ctypes.c_int), ctypes.c_size_t]),
    ("ipm_get_tuning", ctypes.c_int, [_vp, _P(ctypes.c_int), _P(ctypes.c_float), _P(ctypes.c_float)]),
    ("ipm_set_max_level", ctypes.c_int, [_vp, ctypes.c_int]),
    ("ipm_oneshot_retarded", ctypes.c_int, [_vp, _P(ctypes.c_int), _dp, ctypes.c_int, ctypes.c_double, ctypes.c_int64,
                                            _P(ipm_stats)]),
    ("ipm_set_moments_device", ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
    ("ipm_get_moments_device", ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
    ("ipm_dual_solve", ctypes.c_int, [_vp, _P(ipm_stats)]),
    ("ipm_update", ctypes.c_int, [_vp, ctypes.c_double]),
    ("ipm_assemble_hessian", ctypes.c_int, [_vp, _dp, ctypes.c_size_t]),
    ("ipm_factor_hessian", ctypes.c_int, [_vp, _dp, ctypes.c_size_t]),
    ("ipm_step", ctypes.c_int, [_vp, _P(ipm_stats)]),
    ("ipm_run", ctypes.c_int, [_vp, ctypes.c_int64, _P(ipm_stats)]),
    ("ipm_oneshot_step", ctypes.c_int, [_vp, _P(ipm_stats)]),
    ("ipm_sync_stats", ctypes.c_int, [_vp, _P(ipm_stats)]),
    ("ipm_step_timing", ctypes.c_int, [_vp, _P(ctypes.c_float), _P(ctypes.c_float), _P(ctypes.c_float)]),
    ("ipm_dual_solve_noalloc", ctypes.c_int, [ctypes.c_int, ctypes.c_double, _P(ipm_basis), _P(ipm_quadrature),
                                              _P(ipm_entropy), _P(ipm_options), ctypes.c_int, _vp, _vp, _vp,
                                              _vp, _vp, _vp, _P(ipm_stats)]),
    ("ipm_footprint", ctypes.c_int, [_P(ipm_problem), _P(ipm_basis), _P(ipm_quadrature), _P(ipm_entropy),
                                     _P(ipm_options), _P(ctypes.c_size_t)]),
    ("ipm_server_create", ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, _P(_vp)]),
    ("ipm_submit", ctypes.c_int, [_vp, _P(ipm_request), _P(ctypes.c_uint64)]),
    ("ipm_poll", ctypes.c_int, [_vp, ctypes.c_uint64, _P(ipm_result), _dp, ctypes.c_size_t]),
    ("ipm_server_drain", ctypes.c_int, [_vp, ctypes.c_double]),
    ("ipm_server_destroy", None, [_vp]),
    ("ipm_tables", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                  _P(ctypes.c_int), _dp, _dp, _dp, _P(ctypes.c_int), _P(ctypes.c_int)]),
    ("ipm_tables_cc", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     _P(ctypes.c_int), _dp, _dp, _dp, _P(ctypes.c_int), _P(ctypes.c_int)]),
    ("ipm_sc_init", ctypes.c_int, [_P(ipm_problem), _P(ipm_basis), _P(ipm_quadrature), ctypes.c_double, _P(_vp)]),
    ("ipm_sc_step", ctypes.c_int, [_vp, _P(ipm_sc_stats)]),
    ("ipm_sc_run", ctypes.c_int, [_vp, ctypes.c_int64, _P(ipm_sc_stats)]),
    ("ipm_sc_get_nodal", ctypes.c_int, [_vp, _dp, ctypes.c_size_t]),
    ("ipm_sc_get_moments", ctypes.c_int, [_vp, _dp, ctypes.c_size_t]),
    ("ipm_sc_get_node_info", ctypes.c_int, [_vp, _P(ctypes.c_int64), _dp, _dp, ctypes.c_size_t]),
    ("ipm_sc_get_dims", ctypes.c_int, [_vp, _P(ctypes.c_int), _P(ctypes.c_int), _P(ctypes.c_int), _P(ctypes.c_int)]),
    ("ipm_sc_last_error", ctypes.c_char_p, [_vp]),
    ("ipm_sc_destroy", None, [_vp]),
]


def lib():
    """Load libipm.so (built in-tree by __graft_entry__.build()); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libipm.so not found at {LIB_PATH}: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(call, status, ctx=None):
    if status != IPM_OK:
        msg = lib().ipm_last_error(ctx)
        raise IpmError(call, status, msg.decode() if msg else "")


def _dptr(a):
    return a.ctypes.data_as(_dp)


def default_options(precision="fp64", **kw):
    o = ipm_options()
    lib().ipm_default_options(ctypes.byref(o))
    o.precision = PRECISION[precision]
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def ipm_tables(p, total_degree, n_per_dim):
    """Host-only tables of the library: (indices (N,p), nodes (Q,p), weights (Q,), Phi (Q,N))."""
    N = ctypes.c_int()
    Q = ctypes.c_int()
    # size query: with zero capacity the call returns IPM_EINVAL but fills N and Q
    lib().ipm_tables(p, total_degree, n_per_dim, 0, 0, None, None, None, None, ctypes.byref(N), ctypes.byref(Q))
    n, q = N.value, Q.value
    idx = np.zeros((n, p), dtype=np.int32)
    nodes = np.zeros((q, p))
    w = np.zeros(q)
    phi = np.zeros((q, n))
    _check("ipm_tables", lib().ipm_tables(p, total_degree, n_per_dim, n, q, idx.ctypes.data_as(_P(ctypes.c_int)),
                                          _dptr(nodes), _dptr(w), _dptr(phi), ctypes.byref(N), ctypes.byref(Q)))
    return idx, nodes, w, phi


def ipm_tables_cc(p, total_degree, kmax):
    """Host-only nested Clenshaw-Curtis tables: (indices, nodes (Q,p), level weights (kmax+1, Q), Phi (Q,N))."""
    N = ctypes.c_int()
    Q = ctypes.c_int()
    lib().ipm_tables_cc(p, total_degree, kmax, 0, 0, None, None, None, None, ctypes.byref(N), ctypes.byref(Q))
    n, q = N.value, Q.value
    idx = np.zeros((n, p), dtype=np.int32)
    nodes = np.zeros((q, p))
    w = np.zeros((kmax + 1, q))
    phi = np.zeros((q, n))
    _check("ipm_tables_cc", lib().ipm_tables_cc(p, total_degree, kmax, n, q, idx.ctypes.data_as(_P(ctypes.c_int)),
                                                _dptr(nodes), _dptr(w), _dptr(phi), ctypes.byref(N), ctypes.byref(Q)))
    return idx, nodes, w, phi


def ipm_dual_solve_noalloc(kind, gamma, p, total_degree, n_per_dim, entropy, n_cells, d_uhat, d_lam, d_nodal,
                           d_iters, d_status, stream=0, u_minus=0.0, u_plus=0.0, options=None):
    """Dual solve on caller-owned device buffers (integer device addresses); allocates nothing.
    Returns the ipm_stats of the call (the call waits for the solve)."""
    b = ipm_basis(p, total_degree)
    q = _quad(n_per_dim)
    e = ipm_entropy(ENTROPY[entropy], u_minus, u_plus)
    o = options if options is not None else default_options()
    s = ipm_stats()
    _check("ipm_dual_solve_noalloc",
           lib().ipm_dual_solve_noalloc(PROBLEM[kind], gamma, ctypes.byref(b), ctypes.byref(q), ctypes.byref(e),
                                        ctypes.byref(o), n_cells, _vp(d_uhat), _vp(d_lam), _vp(d_nodal), _vp(d_iters),
                                        _vp(d_status), _vp(stream) if stream else None, ctypes.byref(s)))
    return s


def make_problem(kind, nx, x_lo, x_hi, bc=("outflow", "outflow"), cfl=0.5, t_end=0.0, gamma=1.4,
                 x0=0.5, dx0=(0, 0, 0), left=(0, 0, 0, 0), dleft=None, right=(0, 0, 0, 0), dright=None):
    pr = ipm_problem()
    pr.kind = PROBLEM[kind]
    pr.nx, pr.ny = nx, 1
    pr.x_lo, pr.x_hi = x_lo, x_hi
    pr.bc_left, pr.bc_right = BC[bc[0]], BC[bc[1]]
    pr.cfl, pr.t_end, pr.gamma = cfl, t_end, gamma
    pr.ic_kind = 0
    pr.ic_x0 = x0
    for d in range(3):
        pr.ic_dx0[d] = dx0[d]
    for v in range(4):
        pr.ic_left[v] = left[v] if v < len(left) else 0.0
        pr.ic_right[v] = right[v] if v < len(right) else 0.0
        for d in range(3):
            pr.ic_dleft[v][d] = dleft[v][d] if dleft is not None and v < len(dleft) else 0.0
            pr.ic_dright[v][d] = dright[v][d] if dright is not None and v < len(dright) else 0.0
    return pr


def make_problem_2d(nx, ny, x_lo, x_hi, y_lo, y_hi, sides=("periodic",) * 4, mesh="cartesian", ramp_x0=0.0,
                    ramp_deg=0.0, cfl=0.4, t_end=0.0, gamma=1.4, ic="freestream", param=(0, 0, 0, 0), dparam=None,
                    x0=0.5, left=(0, 0, 0, 0), dleft=None, right=(0, 0, 0, 0), dright=None, dx0=(0, 0, 0)):
    """2-D Euler problem; sides = (left, right, bottom, top)."""
    pr = make_problem("euler2d", nx, x_lo, x_hi, bc=sides[:2], cfl=cfl, t_end=t_end, gamma=gamma, x0=x0, dx0=dx0,
                      left=left, dleft=dleft, right=right, dright=dright)
    pr.ny = ny
    pr.y_lo, pr.y_hi = y_lo, y_hi
    pr.bc_bottom, pr.bc_top = BC[sides[2]], BC[sides[3]]
    pr.mesh_kind = MESH[mesh]
    pr.ramp_x0, pr.ramp_deg = ramp_x0, ramp_deg
    pr.ic_kind = IC[ic]
    for v in range(4):
        pr.ic_param[v] = param[v]
        for d in range(3):
            pr.ic_dparam[v][d] = dparam[v][d] if dparam is not None and v < len(dparam) else 0.0
    return pr


class Context:
    """One resident IPM problem on the current CUDA device (wraps ipm_ctx*)."""

    def __init__(self, problem, p, total_degree, n_per_dim, entropy, u_minus=0.0, u_plus=0.0, options=None):
        b = ipm_basis(p, total_degree)
        q = _quad(n_per_dim)
        e = ipm_entropy(ENTROPY[entropy], u_minus, u_plus)
        o = options if options is not None else default_options()
        h = _vp()
        _check("ipm_init", lib().ipm_init(ctypes.byref(problem), ctypes.byref(b), ctypes.byref(q), ctypes.byref(e),
                                          ctypes.byref(o), ctypes.byref(h)))
        self.h = h
        d = ipm_dims()
        _check("ipm_get_dims", lib().ipm_get_dims(self.h, ctypes.byref(d)), self.h)
        self.dims = d
        self.shape = (d.n_cells, d.N, d.m)

    def close(self):
        if self.h:
            lib().ipm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _get(self, fn, shape, out=None):
        """Copy device state into out (a C-contiguous float64 array of this shape, e.g. in pinned memory,
        written in place) or into a new array."""
        if out is None:
            out = np.empty(shape)
        elif out.dtype != np.float64 or not out.flags.c_contiguous or out.size != int(np.prod(shape)):
            raise ValueError(f"{fn}: out must be a C-contiguous float64 array of {int(np.prod(shape))} elements")
        _check(fn, getattr(lib(), fn)(self.h, _dptr(out), out.size), self.h)
        return out

    def _set(self, fn, arr):
        a = np.ascontiguousarray(arr, dtype=np.float64).reshape(self.shape)
        _check(fn, getattr(lib(), fn)(self.h, _dptr(a), a.size), self.h)

    def get_moments(self, out=None):
        return self._get("ipm_get_moments", self.shape, out)

    def set_moments(self, a):
        self._set("ipm_set_moments", a)

    def get_duals(self, out=None):
        return self._get("ipm_get_duals", self.shape, out)

    def set_duals(self, a):
        self._set("ipm_set_duals", a)

    def set_state(self, moments, duals, levels=None, clock=None):
        """Restore moments and duals (C-contiguous float64 arrays of the state's shape are used in place,
        e.g. pinned buffers), and optionally the levels (adaptive contexts) and the clock (ipm_clock)."""
        m = np.ascontiguousarray(moments, dtype=np.float64).reshape(self.shape)
        d = np.ascontiguousarray(duals, dtype=np.float64).reshape(self.shape)
        lv = None if levels is None else np.ascontiguousarray(levels, dtype=np.int32)
        _check("ipm_set_state", lib().ipm_set_state(
            self.h, _dptr(m), _dptr(d), None if lv is None else lv.ctypes.data_as(_P(ctypes.c_int)),
            None if clock is None else ctypes.byref(clock), m.size), self.h)

    def get_state(self, moments=None, duals=None, levels=False, clock=False):
        """(moments, duals[, levels][, clock]); given arrays (C-contiguous float64 of the state's shape)
        are filled in place. levels=True / clock=True also return the level of every cell (adaptive
        contexts) and the ipm_clock."""
        m = np.empty(self.shape) if moments is None else moments
        d = np.empty(self.shape) if duals is None else duals
        for a in (m, d):
            if a.dtype != np.float64 or not a.flags.c_contiguous or a.size != int(np.prod(self.shape)):
                raise ValueError("get_state: arrays must be C-contiguous float64 of the state's shape")
        lv = np.zeros(self.dims.n_cells, dtype=np.int32) if levels else None
        ck = ipm_clock() if clock else None
        _check("ipm_get_state", lib().ipm_get_state(
            self.h, _dptr(m), _dptr(d), None if lv is None else lv.ctypes.data_as(_P(ctypes.c_int)),
            None if ck is None else ctypes.byref(ck), m.size), self.h)
        out = (m, d)
        if levels:
            out += (lv,)
        if clock:
            out += (ck,)
        return out

    def get_nodal_states(self):
        d = self.dims
        return self._get("ipm_get_nodal_states", (d.n_cells, d.m, d.Q))

    def set_max_level(self, level):
        _check("ipm_set_max_level", lib().ipm_set_max_level(self.h, level), self.h)

    def oneshot_retarded(self, max_levels, tolerances, tol, max_steps):
        """Algorithm 4; returns the ipm_stats of the last step."""
        lv = (ctypes.c_int * len(max_levels))(*max_levels)
        tl = (ctypes.c_double * max(1, len(tolerances)))(*tolerances)
        s = ipm_stats()
        _check("ipm_oneshot_retarded", lib().ipm_oneshot_retarded(self.h, lv, tl, len(max_levels), tol, max_steps,
                                                                  ctypes.byref(s)), self.h)
        return s

    def tuning(self):
        """(kernel variant 1 = CTA per cell / 2 = warp per cell, ms of the CTA trial, ms of the warp trial)."""
        k, a, b = ctypes.c_int(), ctypes.c_float(), ctypes.c_float()
        _check("ipm_get_tuning", lib().ipm_get_tuning(self.h, ctypes.byref(k), ctypes.byref(a), ctypes.byref(b)), self.h)
        return k.value, a.value, b.value

    def get_levels(self):
        out = np.empty(self.dims.n_cells, dtype=np.int32)
        _check("ipm_get_levels", lib().ipm_get_levels(self.h, out.ctypes.data_as(_P(ctypes.c_int)), out.size), self.h)
        return out

    def set_moments_device(self, ptr, count):
        _check("ipm_set_moments_device", lib().ipm_set_moments_device(self.h, _vp(ptr), count), self.h)

    def get_moments_device(self, ptr, count):
        _check("ipm_get_moments_device", lib().ipm_get_moments_device(self.h, _vp(ptr), count), self.h)

    def set_stream(self, stream_ptr):
        """Order this context's work on a cudaStream_t given as an integer handle (0 = legacy default)."""
        _check("ipm_set_stream", lib().ipm_set_stream(self.h, _vp(stream_ptr) if stream_ptr else None), self.h)

    def _stats_call(self, fn, *args, sync=True):
        s = ipm_stats()
        _check(fn, getattr(lib(), fn)(self.h, *args, ctypes.byref(s) if sync else None), self.h)
        return s if sync else None

    def dual_solve(self, sync=True):
        return self._stats_call("ipm_dual_solve", sync=sync)

    def assemble_hessian(self):
        """Packed lower-triangular Hessians at the current duals, (n_interior, NM(NM+1)/2)."""
        d = self.dims
        nm = d.N * d.m
        return self._get("ipm_assemble_hessian", (d.n_interior, nm * (nm + 1) // 2))

    def factor_hessian(self):
        """Packed lower-triangular Cholesky factors of those Hessians, (n_interior, NM(NM+1)/2)."""
        d = self.dims
        nm = d.N * d.m
        return self._get("ipm_factor_hessian", (d.n_interior, nm * (nm + 1) // 2))

    def update(self, dt):
        _check("ipm_update", lib().ipm_update(self.h, dt), self.h)

    def step(self, sync=True):
        return self._stats_call("ipm_step", sync=sync)

    def oneshot_step(self, sync=True):
        return self._stats_call("ipm_oneshot_step", sync=sync)

    def run(self, max_steps=2 ** 62):
        return self._stats_call("ipm_run", ctypes.c_int64(max_steps))

    def sync_stats(self):
        return self._stats_call("ipm_sync_stats")

    def step_timing(self):
        """(newton_ms, update_ms, total_ms) of the last step, from events inside its graph."""
        a, b, t = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
        _check("ipm_step_timing", lib().ipm_step_timing(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(t)), self.h)
        return a.value, b.value, t.value


def make_request(problem, p, total_degree, n_per_dim, entropy, u_minus=0.0, u_plus=0.0, options=None, max_steps=2 ** 62):
    r = ipm_request()
    r.problem = problem
    r.basis = ipm_basis(p, total_degree)
    r.quad = _quad(n_per_dim)
    r.entropy = ipm_entropy(ENTROPY[entropy], u_minus, u_plus)
    r.options = options if options is not None else default_options()
    r.max_steps = max_steps
    return r


def footprint(req):
    """Device bytes ipm_init would allocate for the request's problem."""
    b = ctypes.c_size_t()
    _check("ipm_footprint", lib().ipm_footprint(ctypes.byref(req.problem), ctypes.byref(req.basis),
                                                ctypes.byref(req.quad), ctypes.byref(req.entropy),
                                                ctypes.byref(req.options), ctypes.byref(b)))
    return b.value


class Server:
    """Continuous-batching request server (wraps ipm_server*)."""

    def __init__(self, mem_cap_bytes=0, max_active=16):
        h = _vp()
        _check("ipm_server_create", lib().ipm_server_create(mem_cap_bytes, max_active, ctypes.byref(h)))
        self.h = h

    def submit(self, req):
        t = ctypes.c_uint64()
        _check("ipm_submit", lib().ipm_submit(self.h, ctypes.byref(req), ctypes.byref(t)))
        return t.value

    def poll(self, ticket, fetch=True):
        """None while the request runs; else (ipm_result, moments or None). Fetching releases the ticket."""
        r = ipm_result()
        st = lib().ipm_poll(self.h, ticket, ctypes.byref(r), None, 0)
        if st == 8:
            return None
        _check("ipm_poll", st)
        if not fetch or r.status != 0:
            return r, None
        d = r.dims
        out = np.empty((d.n_cells, d.N, d.m))
        _check("ipm_poll", lib().ipm_poll(self.h, ticket, None, _dptr(out), out.size))
        return r, out

    def drain(self, timeout_s=600.0):
        _check("ipm_server_drain", lib().ipm_server_drain(self.h, timeout_s))

    def close(self):
        if self.h:
            lib().ipm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Collocation:
    """Stochastic Collocation on the GPU (ipm_sc_*): one deterministic run per quadrature node with the
    IPM update's flux, each node on its own time steps; see include/ipm.h."""

    def __init__(self, problem, p, total_degree, n_per_dim, steady_tol=0.0):
        import numpy as np  # noqa: F401
        self.h = None
        h = _vp()
        b = ipm_basis(p=p, total_degree=total_degree)
        q = _quad(n_per_dim)
        st = lib().ipm_sc_init(ctypes.byref(problem), ctypes.byref(b), ctypes.byref(q), float(steady_tol),
                               ctypes.byref(h))
        if st != IPM_OK:
            msg = lib().ipm_sc_last_error(None)
            raise IpmError("ipm_sc_init", st, msg.decode() if msg else "")
        self.h = h
        c, n, N, m = (ctypes.c_int() for _ in range(4))
        lib().ipm_sc_get_dims(self.h, ctypes.byref(c), ctypes.byref(n), ctypes.byref(N), ctypes.byref(m))
        self.n_cells, self.Q, self.N, self.m = c.value, n.value, N.value, m.value

    def _check(self, call, st):
        if st != IPM_OK:
            msg = lib().ipm_sc_last_error(self.h)
            raise IpmError(call, st, msg.decode() if msg else "")

    def close(self):
        if self.h:
            lib().ipm_sc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self):
        s = ipm_sc_stats()
        self._check("ipm_sc_step", lib().ipm_sc_step(self.h, ctypes.byref(s)))
        return s

    def run(self, max_steps=2 ** 62):
        s = ipm_sc_stats()
        self._check("ipm_sc_run", lib().ipm_sc_run(self.h, int(max_steps), ctypes.byref(s)))
        return s

    def get_nodal(self):
        import numpy as np
        a = np.empty((self.n_cells, self.Q, self.m))
        self._check("ipm_sc_get_nodal", lib().ipm_sc_get_nodal(self.h, _dptr(a), a.size))
        return a

    def get_moments(self):
        import numpy as np
        a = np.empty((self.n_cells, self.N, self.m))
        self._check("ipm_sc_get_moments", lib().ipm_sc_get_moments(self.h, _dptr(a), a.size))
        return a

    def node_info(self):
        """(steps, t, residual) per node."""
        import numpy as np
        n = np.empty(self.Q, dtype=np.int64)
        t = np.empty(self.Q)
        r = np.empty(self.Q)
        self._check("ipm_sc_get_node_info", lib().ipm_sc_get_node_info(
            self.h, n.ctypes.data_as(_P(ctypes.c_int64)), _dptr(t), _dptr(r), self.Q))
        return n, t, r
