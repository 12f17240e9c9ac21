"""Adaptive IPM (Sec. 5, Algorithm 3) on 2-D meshes (test infrastructure; see ``oracle/__init__``).

Refinement levels l = 0..L-1 are total degrees M_l (consecutive: M_l = M_0 + l) with N_l moments.
In the graded ordering of the multi-indices the moments of level l are the first N_l entries of
the finest level's moment vector, so states are stored at the finest size N_{L-1} with the entries
beyond the cell's level held at zero. One tensor Gauss rule serves every level (exact for the
products of every level), so the nodal states of all cells live on the same nodes.

* Smoothness indicator (Eq. errorIndicator) on the first conserved variable (the density):
  S_l = <(u_l - u_{l-1})^2> / <u_l^2> = sum_{|i| = M_l} u_i^2 / sum_{|i| <= M_l} u_i^2 (orthonormal basis).
* DetermineRefinementLevel: keep l if delta_- <= S_l <= delta_+, go one level down if S_l < delta_-,
  one level up if S_l > delta_+ (clamped to 0..L-1). The paper prints delta_- > delta_+; the
  interval is taken as [min, max] of the two printed values. The indicator is evaluated on the
  cell's moments u_hat^n at its level (Algorithm 3 writes DetermineRefinementLevel(lambda_hat), but
  Eq. errorIndicator is defined on moments).
* Initial level (Algorithm 3: "choose initial refinement level"): the finest-level projection of the
  initial data, lowered one level at a time while the indicator is below delta_-.
* Step n (Algorithm 3): dual solve of every interior cell at its level l^n (Eq.
  dualIterationFunctionAd: Newton with the level's basis, warm-started at lambda^n); new levels l^{n+1}
  from u_hat^n; moment update c (Eq. adaptiveFVUpdate) with every stencil cell evaluated with its
  own level's duals and the result projected onto level l^{n+1}; the duals of the next solve are
  lambda^{n+1} padded with zeros or truncated to l^{n+1}.
* Quadrature per level (Levels.quad_levels; Sec. 5 uses nested rules, Sec. 7 Clenshaw-Curtis levels):
  level l integrates with the nested tensor Clenshaw-Curtis rule of level quad_levels[l] (a prefix of
  the finest rule's nodes, with its own weights; prob.space is then a basis.NestedCCSpace). The dual
  problem of level l uses that rule (Eq. dualIterationFunctionAd, <.>_{Q_l}); the update of a cell
  whose new level is l integrates over Q_l with every stencil cell's ansatz evaluated at those nodes
  (the paper: a coarser neighbour is evaluated at the finer nodes); the time step takes the wave
  speed of each interior cell at the nodes of its new level and of each Dirichlet ghost at the nodes
  of its own level; the initial moments and duals are projected with the rule of the initial level.
  Without quad_levels every level shares the one rule of prob.space.

Pinned by: tests/test_oracle_adaptive.py (indicator against its integral definition on the nodes,
level rules, a single level reproducing the fixed-degree scheme, pad/truncate bookkeeping,
conservation on periodic meshes).
"""
from dataclasses import dataclass

import numpy as np

from . import dual as dualmod
from . import scheme2d as s2


class SubSpace:
    """The first N_l basis functions of a space (same nodes and weights)."""

    def __init__(self, space, n):
        self.N = n
        self.Q = space.Q
        self.w = space.w
        self.nodes = space.nodes
        self.Phi = space.Phi[:, :n]

    def project(self, values_at_nodes):
        return np.einsum("k,...ka,ki->...ia", self.w, values_at_nodes, self.Phi)

    def evaluate(self, coeffs):
        return np.einsum("ki,...ia->...ka", self.Phi, coeffs)


@dataclass
class Levels:
    degrees: tuple          # consecutive total degrees, coarsest first
    delta_lo: float
    delta_hi: float
    quad_levels: tuple = None   # Clenshaw-Curtis level of every refinement level (nested rules), or None


def level_space(prob, lv: Levels, l: int):
    """Basis and quadrature of refinement level l: the first N_l basis functions with the shared rule,
    or with the level's nested Clenshaw-Curtis rule."""
    nl, _ = level_sizes(prob.space, lv)
    if lv.quad_levels is None:
        return SubSpace(prob.space, nl[l])
    return prob.space.level(lv.quad_levels[l], nl[l])


def level_nodes(prob, lv: Levels):
    """Q_l of every refinement level."""
    if lv.quad_levels is None:
        return [prob.space.Q] * len(lv.degrees)
    return [prob.space.level_q(k) for k in lv.quad_levels]


def indicator(uhat0, n_l, n_prev):
    """S_l of Eq. errorIndicator on one variable: uhat0 (..., N) moments, level sizes N_l and N_{l-1}."""
    idx = np.arange(uhat0.shape[-1])
    top = np.sum(np.where((idx >= n_prev) & (idx < n_l), uhat0 ** 2, 0.0), axis=-1)
    tot = np.sum(np.where(idx < n_l, uhat0 ** 2, 0.0), axis=-1)
    return top / tot


def level_sizes(space, lv: Levels):
    """(N_l, N_{l-1}) per level; N_{-1} counts the moments of degree below the coarsest level's."""
    deg = np.sum(space.indices, axis=1)
    nl = [int(np.sum(deg <= M)) for M in lv.degrees]
    nprev = [int(np.sum(deg <= M - 1)) for M in lv.degrees]
    return nl, nprev


def _indicator_levels(uhat, level, nl, nprev):
    n_cur = np.asarray(nl)[level]
    n_prv = np.asarray(nprev)[level]
    return indicator(uhat[..., 0], n_cur[..., None], n_prv[..., None])


def new_levels(uhat, level, nl, nprev, lv: Levels):
    S = _indicator_levels(uhat, level, nl, nprev)
    lo, hi = min(lv.delta_lo, lv.delta_hi), max(lv.delta_lo, lv.delta_hi)
    new = np.where(S < lo, level - 1, np.where(S > hi, level + 1, level))
    return np.clip(new, 0, len(nl) - 1), S


def truncate(arr, level, nl):
    """Zero the moments beyond each cell's level: arr (..., N, m), level (...)."""
    idx = np.arange(arr.shape[-2])
    keep = idx[None, :] < np.asarray(nl)[level][..., None]
    return np.where(keep[..., None], arr, 0.0)


@dataclass
class AdaptiveState:
    uhat: np.ndarray        # (ny+2, nx+2, N_max, m)
    lam: np.ndarray
    level: np.ndarray       # (ny+2, nx+2) int
    t: float = 0.0
    n: int = 0
    last_dt: float = 0.0
    newton_iters: np.ndarray = None
    newton_status: np.ndarray = None
    residual: float = np.inf


def initial_state(prob: s2.Problem2D, lv: Levels) -> AdaptiveState:
    """Finest projection, levels lowered while the indicator is below delta_-, then truncated; every
    cell, ghosts included, gets a level. Dirichlet ghosts then converge their duals at their level."""
    st = s2.initial_state(prob)
    nl, nprev = level_sizes(prob.space, lv)
    level = np.full(st.uhat.shape[:2], len(nl) - 1, dtype=np.int64)
    lo = min(lv.delta_lo, lv.delta_hi)
    for _ in range(len(nl)):
        S = _indicator_levels(st.uhat, level, nl, nprev)
        level = np.where((S < lo) & (level > 0), level - 1, level)
    if lv.quad_levels is None:
        out = AdaptiveState(uhat=truncate(st.uhat, level, nl), lam=truncate(st.lam, level, nl), level=level)
    else:
        # the initial level's own rule: u_j^0 = <u_IC phi_l>_{Q_l} (Algorithm 3, first loop)
        ny, nx = prob.mesh.ny, prob.mesh.nx
        ubar = prob.ic.cell_states(prob.phys, prob.mesh, prob.space.nodes, ny + 2, nx + 2)
        gs = prob.ent.grad_s(ubar)
        uhat, lam = np.zeros_like(st.uhat), np.zeros_like(st.lam)
        for l, n in enumerate(nl):
            sel = np.nonzero(level == l)
            V = level_space(prob, lv, l)
            uhat[sel[0], sel[1], :n] = V.project(ubar[sel][:, :V.Q])
            lam[sel[0], sel[1], :n] = V.project(gs[sel][:, :V.Q])
        out = AdaptiveState(uhat=uhat, lam=lam, level=level)
    d = s2._dirichlet_mask(prob)
    for l, n in enumerate(nl):
        sel = np.nonzero(d & (level == l))
        if sel[0].size:
            li, _, stat, _ = dualmod.dual_solve(level_space(prob, lv, l), prob.ent, out.lam[sel][:, :n],
                                                out.uhat[sel][:, :n], prob.newton)
            assert np.all(stat == 0)
            lam_sel = out.lam[sel]
            lam_sel[:, :n] = li
            out.lam[sel] = lam_sel
    return out


def _time_step_and_update(prob, lv: Levels, st: AdaptiveState, lam, level, clip):
    """dt of the step and the new moments (Eq. adaptiveFVUpdate) of the interior cells at their new
    levels (level: new levels of the interior, the ghosts' own levels)."""
    nl, _ = level_sizes(prob.space, lv)
    U = s2.nodal_states(prob, lam)                  # every cell's ansatz at all nodes of prob.space
    uhat = st.uhat.copy()
    if lv.quad_levels is None:
        dt = s2.time_step(prob, U, st.t, clip=clip)
        uhat[1:-1, 1:-1] = truncate(s2.moment_update(prob, lam, dt), level[1:-1, 1:-1], nl)
        return dt, uhat
    # wave speeds at the nodes of each cell's (new) level; interior and Dirichlet ghosts
    qn = np.asarray(level_nodes(prob, lv))[level]                    # (ny+2, nx+2)
    cells = s2._dirichlet_mask(prob)
    cells[1:-1, 1:-1] = True
    speed = prob.phys.speed(U)                                       # (ny+2, nx+2, Q)
    at = np.arange(U.shape[-2])[None, None, :] < qn[..., None]
    smax = float(np.max(np.where(at & cells[..., None], speed, 0.0)))
    dt = prob.cfl * prob.mesh.h_min() / smax
    if clip and prob.t_end > 0 and st.t + dt > prob.t_end:
        dt = prob.t_end - st.t
    inner = s2.nodal_update(prob, U, dt)                             # (ny, nx, Q, m), every node
    new = np.zeros(uhat[1:-1, 1:-1].shape)
    for l, n in enumerate(nl):
        sel = np.nonzero(level[1:-1, 1:-1] == l)
        if sel[0].size:
            V = level_space(prob, lv, l)
            new[sel[0], sel[1], :n] = V.project(inner[sel][:, :V.Q])
    uhat[1:-1, 1:-1] = new
    return dt, uhat


def ipm_step(prob: s2.Problem2D, st: AdaptiveState, lv: Levels) -> AdaptiveState:
    """One time step of Algorithm 3 on the interior cells."""
    nl, nprev = level_sizes(prob.space, lv)
    ny, nx = prob.mesh.ny, prob.mesh.nx
    lam = st.lam.copy()
    it = np.zeros((ny, nx), dtype=np.int64)
    stat = np.zeros((ny, nx), dtype=np.int64)
    inner_level = st.level[1:-1, 1:-1]
    for l, n in enumerate(nl):
        sel = np.nonzero(inner_level == l)
        if sel[0].size == 0:
            continue
        sub = level_space(prob, lv, l)
        jj, ii = sel[0] + 1, sel[1] + 1
        li, itl, sl, _ = dualmod.dual_solve(sub, prob.ent, st.lam[jj, ii, :n], st.uhat[jj, ii, :n], prob.newton)
        lam[jj, ii, :n] = li
        it[sel] = itl
        stat[sel] = sl
    level = st.level.copy()
    level[1:-1, 1:-1], _ = new_levels(st.uhat[1:-1, 1:-1], inner_level, nl, nprev, lv)
    # periodic ghosts mirror the levels of the cells they copy (they are never read by the update)
    dt, uhat = _time_step_and_update(prob, lv, st, lam, level, clip=True)
    lam_next = lam.copy()
    lam_next[1:-1, 1:-1] = truncate(lam[1:-1, 1:-1], level[1:-1, 1:-1], nl)
    res = s2.steady_residual(prob, uhat, st.uhat)
    return AdaptiveState(uhat=uhat, lam=lam_next, level=level, t=st.t + dt, n=st.n + 1, last_dt=dt,
                         newton_iters=it, newton_status=stat, residual=res)


def cap_levels(st: AdaptiveState, cap: int, nl) -> AdaptiveState:
    """Lower every interior level above cap to cap and truncate its moments and duals (the ghost cells
    keep their initial levels)."""
    level = st.level.copy()
    level[1:-1, 1:-1] = np.minimum(level[1:-1, 1:-1], cap)
    return AdaptiveState(uhat=truncate(st.uhat, level, nl), lam=truncate(st.lam, level, nl), level=level, t=st.t,
                         n=st.n, last_dt=st.last_dt, residual=st.residual)


def oneshot_step(prob: s2.Problem2D, st: AdaptiveState, lv: Levels, cap: int) -> AdaptiveState:
    """One pseudo-time step of Algorithm 4 (adaptive One-Shot IPM): one damped Newton step per interior
    cell at its level l^n (Eq. dualIterationFunctionAd), new levels from u_hat^n limited by the current
    maximal level cap, moment update projected onto the new levels, steady residual.

    Reading: Algorithm 4 prints max{DetermineRefinementLevel, l*_l}; the text describes l*_l as the
    maximal refinement level of the current stage, so the level is min{DetermineRefinementLevel, l*_l}."""
    nl, nprev = level_sizes(prob.space, lv)
    ny, nx = prob.mesh.ny, prob.mesh.nx
    lam = st.lam.copy()
    it = np.zeros((ny, nx), dtype=np.int64)
    stat = np.zeros((ny, nx), dtype=np.int64)
    inner_level = st.level[1:-1, 1:-1]
    for l, n in enumerate(nl):
        sel = np.nonzero(inner_level == l)
        if sel[0].size == 0:
            continue
        sub = level_space(prob, lv, l)
        jj, ii = sel[0] + 1, sel[1] + 1
        li, itl, sl, _ = dualmod.dual_solve(sub, prob.ent, st.lam[jj, ii, :n], st.uhat[jj, ii, :n], prob.newton,
                                            one_step=True)
        lam[jj, ii, :n] = li
        it[sel] = itl
        stat[sel] = sl
    level = st.level.copy()
    new, _ = new_levels(st.uhat[1:-1, 1:-1], inner_level, nl, nprev, lv)
    level[1:-1, 1:-1] = np.minimum(new, cap)
    dt, uhat = _time_step_and_update(prob, lv, st, lam, level, clip=False)
    lam_next = lam.copy()
    lam_next[1:-1, 1:-1] = truncate(lam[1:-1, 1:-1], level[1:-1, 1:-1], nl)
    res = s2.steady_residual(prob, uhat, st.uhat)
    return AdaptiveState(uhat=uhat, lam=lam_next, level=level, t=st.t + dt, n=st.n + 1, last_dt=dt,
                         newton_iters=it, newton_status=stat, residual=res)


def oneshot_retarded(prob: s2.Problem2D, lv: Levels, caps, tolerances, tol, max_steps):
    """Algorithm 4: refinement retardation. Stage l allows levels up to caps[l]; the stage advances when
    the steady residual falls below tolerances[l]; the run stops at residual tol (once the last stage
    is reached) or after max_steps. Returns (state, [(step, residual, stage)])."""
    nl, _ = level_sizes(prob.space, lv)
    stage = 0
    st = cap_levels(initial_state(prob, lv), caps[0], nl)
    hist = []
    while st.n < max_steps:
        st = oneshot_step(prob, st, lv, caps[stage])
        hist.append((st.n, st.residual, stage))
        if stage + 1 < len(caps) and st.residual < tolerances[stage]:
            stage += 1
        elif stage + 1 == len(caps) and st.residual < tol:
            break
    return st, hist
