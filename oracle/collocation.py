"""Stochastic Collocation (SC), the non-intrusive baseline the paper compares IPM with (test
infrastructure; see ``oracle/__init__``).

SC (Sec. 2, the collocation paragraph; Sec. 7, the IPM-versus-SC comparisons) runs the deterministic
solver once per quadrature node xi_k, independently, and takes the moments from the quadrature rule:
  u_hat_i = sum_k w_k u(x, t, xi_k) phi_i(xi_k).
Here the deterministic solver is the finite-volume scheme of the IPM update with the same numerical
flux, applied to the nodal state of one node (scheme1d.nodal_update / scheme2d.nodal_update with a
node axis of length one):
* initial state: the exact nodal cell averages of the initial data (the values IPM projects);
* boundary conditions as in the IPM schemes (outflow, periodic, Dirichlet ghosts, slip walls);
* time step per node (a black-box run knows nothing of the other nodes): dt_k = CFL h / s_max,k with
  s_max,k the largest wave speed of node k over the same cells as the IPM time step; in 1-D the
  Lax-Friedrichs viscosity dx/(2 dt_k) uses the node's own step;
* unsteady problems (t_end > 0): each node steps until t_k >= t_end, the last step clipped to t_end;
* steady problems (t_end == 0): each node iterates in pseudo-time until its own residual
  sum_c A_c |rho_c^{n+1} - rho_c^n| (Eq. residualSteady on the node's density; A_c = dx in 1-D)
  falls below the tolerance, as the paper iterates every collocation point to its own threshold.

Pinned by: tests/test_oracle_collocation.py (every node against the independent plain-loop
deterministic solvers of the scheme tests, 1-D and on the ramp mesh; conservation node by node on
periodic meshes; the Burgers expectation against the exact Rankine-Hugoniot solution; a node-
independent initial state reproducing the IPM deterministic limit; steady runs ending below the
tolerance).
"""
from dataclasses import dataclass

import numpy as np

from . import scheme1d as s1
from . import scheme2d as s2


@dataclass
class SCResult:
    U: np.ndarray          # nodal states with ghosts: 1-D (nx+2, Q, m), 2-D (ny+2, nx+2, Q, m)
    steps: np.ndarray      # (Q,) steps taken by every node
    t: np.ndarray          # (Q,) time (pseudo-time) reached by every node
    residual: np.ndarray   # (Q,) last steady residual of every node (inf before the first step)

    def moments(self, space):
        """u_hat = sum_k w_k U_k phi(xi_k): the SC moments, [cells..][N][m]."""
        return space.project(self.U)


def _run_node(u, step, residual, dt_of, t_end, steady_tol, max_steps):
    """One node's black-box run: u has a node axis of length one."""
    t, n, res = 0.0, 0, np.inf
    while n < max_steps:
        if t_end > 0.0:
            if t >= t_end:
                break
        elif res < steady_tol:
            break
        dt = dt_of(u, t)
        new = step(u, dt)
        res = residual(new, u)
        u, t, n = new, t + dt, n + 1
    return u, t, n, res


def initial_nodal_1d(prob: s1.Problem1D) -> np.ndarray:
    U = s1.nodal_cell_averages(prob)
    s1.apply_bc(prob, U)
    return U


def run_1d(prob: s1.Problem1D, steady_tol: float = 0.0, max_steps: int = 10 ** 9, nodes=None) -> SCResult:
    """SC of a 1-D problem: every node of prob.space run on its own (see the module docstring). nodes:
    indices of the nodes to run (default all); the result holds those nodes in that order."""
    U0 = initial_nodal_1d(prob)
    if nodes is not None:
        U0 = U0[:, list(nodes)]
    Q = U0.shape[1]

    def step(u, dt):
        new = u.copy()
        new[1:-1] = s1.nodal_update(prob, u, dt)
        s1.apply_bc(prob, new)
        return new

    residual = lambda new, old: float(np.sum(prob.dx * np.abs(new[1:-1, 0, 0] - old[1:-1, 0, 0])))
    dt_of = lambda u, t: s1.time_step(prob, u, t)
    out = np.empty_like(U0)
    steps, times, res = np.zeros(Q, dtype=np.int64), np.zeros(Q), np.zeros(Q)
    for k in range(Q):
        u, times[k], steps[k], res[k] = _run_node(U0[:, k:k + 1].copy(), step, residual, dt_of, prob.t_end,
                                                  steady_tol, max_steps)
        out[:, k] = u[:, 0]
    return SCResult(U=out, steps=steps, t=times, residual=res)


def initial_nodal_2d(prob: s2.Problem2D) -> np.ndarray:
    ny, nx = prob.mesh.ny, prob.mesh.nx
    return prob.ic.cell_states(prob.phys, prob.mesh, prob.space.nodes, ny + 2, nx + 2)


def run_2d(prob: s2.Problem2D, steady_tol: float = 0.0, max_steps: int = 10 ** 9, nodes=None) -> SCResult:
    """SC of a 2-D problem: every node of prob.space run on its own (see the module docstring). nodes:
    indices of the nodes to run (default all); the result holds those nodes in that order."""
    U0 = initial_nodal_2d(prob)
    if nodes is not None:
        U0 = U0[:, :, list(nodes)]
    Q = U0.shape[2]
    area = prob.mesh.area()

    def step(u, dt):
        new = u.copy()
        new[1:-1, 1:-1] = s2.nodal_update(prob, u, dt)
        return new

    residual = lambda new, old: float(np.sum(area * np.abs(new[1:-1, 1:-1, 0, 0] - old[1:-1, 1:-1, 0, 0])))
    dt_of = lambda u, t: s2.time_step(prob, u, t)
    out = np.empty_like(U0)
    steps, times, res = np.zeros(Q, dtype=np.int64), np.zeros(Q), np.zeros(Q)
    for k in range(Q):
        u, times[k], steps[k], res[k] = _run_node(U0[:, :, k:k + 1].copy(), step, residual, dt_of, prob.t_end,
                                                  steady_tol, max_steps)
        out[:, :, k] = u[:, :, 0]
    return SCResult(U=out, steps=steps, t=times, residual=res)
