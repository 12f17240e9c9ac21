"""IPM finite-volume scheme on 1-D meshes (test infrastructure; see ``oracle/__init__``).

Cells j = 1..nx of width dx on [x_lo, x_hi], plus ghost cells j = 0 and j = nx+1 (Algorithm 1 runs
its dual loop over j = 0..nx+1 and its update over j = 1..nx).

* Initial moments (Algorithm 1, first loop): u_j^0 = (1/dx) int_cell <u_IC(x,.) phi>_Q dx. For the
  piecewise-constant Riemann data used here the cell average at each node is exact:
  frac * U_L(xi) + (1 - frac) * U_R(xi), frac = clip((x0(xi) - x_{j-1/2}) / dx, 0, 1).
* Initial duals (not fixed by the paper): lambda_j^(0) = <grad s(ubar_j(xi)) phi^T>_Q^T, the
  projection of the nodal entropy variables. The dual minimiser is unique, so only the iteration
  count depends on this choice.
* Moment update c (Eq. momentIterationFunction, quadrature form Eq. momentUpQuadrature):
  u_j^{n+1} = sum_k w_k [u_k^(j) - dt/dx (g(u_k^(j), u_k^(j+1)) - g(u_k^(j-1), u_k^(j)))] phi(xi_k)
  with u_k^(j) = u_s(lambda_j^T phi(xi_k)) and g the Lax-Friedrichs flux (or, for comparisons with
  the 2-D scheme, the local Lax-Friedrichs flux of physics.rusanov).
* Time step (not fixed by the paper beyond "CFL"): dt = CFL dx / max_{j,k} speed(u_k^(j)) over all
  cells including ghosts, evaluated at the freshly solved duals; the last step is clipped to t_end.
* Boundary conditions, applied to the initial state and after each update: outflow copies the
  neighbour's moments and duals, periodic wraps, dirichlet keeps the ghost's initial state (its
  duals are converged once at the start).
* Algorithm 1 (IPM): converge the dual problem in every cell (ghosts included), then update.
* Algorithm 2 (One-Shot IPM): one Newton step in every interior cell, ghost duals from the
  boundary condition, then update; the steady residual is
  sum_j dx |u_{0,1,j}^{n+1} - u_{0,1,j}^n| (Eq. residualSteady restricted to the zero-order moment of
  the first conserved variable, as the paper does for the density).

Pinned by: tests/test_oracle_scheme.py (constant states, deterministic limit against a separate
scalar/system LF solver, conservation on periodic grids, SG reduction against the analytic
triple-product flux of App. A, Burgers Rankine-Hugoniot expectation, One-Shot fixed point).
"""
from dataclasses import dataclass, field

import numpy as np

from . import dual as dualmod
from .physics import lax_friedrichs, rusanov


@dataclass
class RiemannIC:
    """Piecewise-constant data with one jump; every parameter affine in xi.

    left/right are conserved-variable functions of xi (callables xi(Q,p) -> (Q,m)); x0 likewise
    returns (Q,).
    """
    left: object
    right: object
    x0: object


@dataclass
class Problem1D:
    phys: object
    ent: object
    space: object
    nx: int
    x_lo: float
    x_hi: float
    ic: RiemannIC
    bc: str = "outflow"           # outflow | periodic | dirichlet, or "left/right" e.g. "dirichlet/outflow"
    cfl: float = 0.5
    t_end: float = 0.0
    newton: dualmod.NewtonOptions = field(default_factory=dualmod.NewtonOptions)
    flux: str = "lf"              # "lf": global Lax-Friedrichs (App. A); "rusanov": local LF (the 2-D flux)

    @property
    def dx(self):
        return (self.x_hi - self.x_lo) / self.nx

    @property
    def bc_sides(self):
        parts = self.bc.split("/")
        return (parts[0], parts[-1])


@dataclass
class State1D:
    uhat: np.ndarray      # (nx+2, N, m)
    lam: np.ndarray       # (nx+2, N, m)
    t: float = 0.0
    n: int = 0
    last_dt: float = 0.0
    newton_iters: np.ndarray = None
    newton_status: np.ndarray = None
    residual: float = np.inf


def nodal_cell_averages(prob: Problem1D) -> np.ndarray:
    """ubar_j(xi_k) for j = 0..nx+1: shape (nx+2, Q, m)."""
    sp = prob.space
    UL = prob.ic.left(sp.nodes)           # (Q, m)
    UR = prob.ic.right(sp.nodes)
    x0 = prob.ic.x0(sp.nodes)             # (Q,)
    j = np.arange(prob.nx + 2)
    x_left = prob.x_lo + (j - 1) * prob.dx     # left edge of cell j (ghost 0 sits left of x_lo)
    frac = np.clip((x0[None, :] - x_left[:, None]) / prob.dx, 0.0, 1.0)   # (nx+2, Q)
    return frac[..., None] * UL[None] + (1.0 - frac[..., None]) * UR[None]


def initial_state(prob: Problem1D) -> State1D:
    ubar = nodal_cell_averages(prob)
    uhat = prob.space.project(ubar)
    lam = prob.space.project(prob.ent.grad_s(ubar))
    apply_bc(prob, uhat)        # outflow / periodic ghosts take their boundary state from the start
    apply_bc(prob, lam)
    st = State1D(uhat=uhat, lam=lam)
    fixed = [g for g, side in zip((0, prob.nx + 1), prob.bc_sides) if side == "dirichlet"]
    if fixed:
        # fixed ghosts: their duals are converged once and then kept
        g = np.array(fixed)
        lg, _, _, _ = dualmod.dual_solve(prob.space, prob.ent, lam[g], uhat[g], prob.newton)
        st.lam[g] = lg
    return st


def apply_bc(prob: Problem1D, arr: np.ndarray) -> None:
    nx = prob.nx
    left, right = prob.bc_sides
    if (left == "periodic") != (right == "periodic"):
        raise ValueError(prob.bc)
    for ghost, inner, wrap, side in ((0, 1, nx, left), (nx + 1, nx, 1, right)):
        if side == "outflow":
            arr[ghost] = arr[inner]
        elif side == "periodic":
            arr[ghost] = arr[wrap]
        elif side != "dirichlet":
            raise ValueError(prob.bc)


def nodal_states(prob: Problem1D, lam: np.ndarray) -> np.ndarray:
    """u_k^(j) = u_s(lambda_j^T phi(xi_k)) for every cell: (C, Q, m)."""
    return prob.ent.u_s(prob.space.evaluate(lam))


def time_step(prob: Problem1D, U: np.ndarray, t: float) -> float:
    smax = float(np.max(prob.phys.speed(U)))
    dt = prob.cfl * prob.dx / smax
    if prob.t_end > 0 and t + dt > prob.t_end:
        dt = prob.t_end - t
    return dt


def nodal_update(prob: Problem1D, U: np.ndarray, dt: float) -> np.ndarray:
    """The finite-volume update of nodal states U (nx+2, Q, m), node by node, for j = 1..nx:
    u_k^(j) - dt/dx (g(u_k^(j), u_k^(j+1)) - g(u_k^(j-1), u_k^(j))): (nx, Q, m)."""
    if prob.flux == "rusanov":
        G = rusanov(prob.phys, U[:-1], U[1:], np.array([1.0]))
    else:
        G = lax_friedrichs(prob.phys, U[:-1], U[1:], prob.dx, dt)   # faces j+1/2, j = 0..nx: (nx+1, Q, m)
    return U[1:-1] - (dt / prob.dx) * (G[1:] - G[:-1])


def moment_update(prob: Problem1D, lam: np.ndarray, dt: float) -> np.ndarray:
    """c(lambda_{j-1}, lambda_j, lambda_{j+1}) for j = 1..nx (Eq. momentUpQuadrature): (nx, N, m)."""
    return prob.space.project(nodal_update(prob, nodal_states(prob, lam), dt))


def ipm_step(prob: Problem1D, st: State1D) -> State1D:
    """One time step of Algorithm 1."""
    lam, it, stat, _ = dualmod.dual_solve(prob.space, prob.ent, st.lam, st.uhat, prob.newton)
    U = nodal_states(prob, lam)
    dt = time_step(prob, U, st.t)
    uhat = st.uhat.copy()
    uhat[1:-1] = moment_update(prob, lam, dt)
    apply_bc(prob, uhat)
    lam_next = lam.copy()
    apply_bc(prob, lam_next)
    return State1D(uhat=uhat, lam=lam_next, t=st.t + dt, n=st.n + 1, last_dt=dt,
                   newton_iters=it, newton_status=stat, residual=steady_residual(prob, uhat, st.uhat))


def steady_residual(prob: Problem1D, uhat_new: np.ndarray, uhat_old: np.ndarray) -> float:
    """Eq. residualSteady on the zero-order moment of the first conserved variable."""
    return float(np.sum(prob.dx * np.abs(uhat_new[1:-1, 0, 0] - uhat_old[1:-1, 0, 0])))


def oneshot_step(prob: Problem1D, st: State1D) -> State1D:
    """One pseudo-time step of Algorithm 2 (One-Shot IPM)."""
    lam = st.lam.copy()
    li, it, stat, _ = dualmod.dual_solve(prob.space, prob.ent, st.lam[1:-1], st.uhat[1:-1], prob.newton,
                                         one_step=True)
    lam[1:-1] = li
    apply_bc(prob, lam)
    U = nodal_states(prob, lam)
    dt = prob.cfl * prob.dx / float(np.max(prob.phys.speed(U)))
    uhat = st.uhat.copy()
    uhat[1:-1] = moment_update(prob, lam, dt)
    apply_bc(prob, uhat)
    res = steady_residual(prob, uhat, st.uhat)
    return State1D(uhat=uhat, lam=lam, t=st.t + dt, n=st.n + 1, last_dt=dt,
                   newton_iters=it, newton_status=stat, residual=res)


def run(prob: Problem1D, max_steps: int = 10 ** 9, state: State1D = None) -> State1D:
    """Algorithm 1 until t_end (or max_steps)."""
    st = initial_state(prob) if state is None else state
    while st.t < prob.t_end and st.n < max_steps:
        st = ipm_step(prob, st)
        if np.any(st.newton_status != 0):
            raise RuntimeError(f"dual solve failed at step {st.n}: {np.bincount(st.newton_status)}")
    return st


def expectation_variance(uhat: np.ndarray):
    """E = u_hat_0 and Var = sum_{i>=1} u_hat_i^2 per variable (Sec. 2; the sum starts after the
    zero-order moment, the printed upper index N is garbled)."""
    return uhat[..., 0, :], np.sum(uhat[..., 1:, :] ** 2, axis=-2)
