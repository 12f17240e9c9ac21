"""IPM finite-volume scheme on structured 2-D quadrilateral meshes (test infrastructure; see
``oracle/__init__``). The 2-D Euler system of Sec. 7 (conserved rho, rho v_1, rho v_2, E).

Mesh: vertices (X[i, j], Y[i, j]), i = 0..nx, j = 0..ny; interior cell (i, j), i < nx, j < ny, has
the corners (i, j), (i+1, j), (i+1, j+1), (i, j+1). Arrays with ghosts are indexed [j+1, i+1]
(shape (ny+2, nx+2, ...)): one ghost layer on every side, corners unused.
* x-face f (f = 0..nx) joins vertices (f, j) and (f, j+1); its unit normal points to increasing i.
* y-face g (g = 0..ny) joins vertices (i, g) and (i+1, g); its unit normal points to increasing j.
* cell area by the shoelace formula.

Moment update of an interior cell c (Eq. momentIterationFunction in quadrature form, Eq.
momentUpQuadrature, with the divergence theorem over the cell's four faces):
  u_c^{n+1} = sum_k w_k [u_k^(c) - dt/A_c sum_faces L_f s_f g(u_k^(in), u_k^(out); n_f)] phi(xi_k)
where g is the local Lax-Friedrichs (Rusanov) flux across the face (physics.rusanov: a mapped mesh
has no single dx for the global form of App. A), (in, out) the cells behind and in front of the
face normal, s_f = +1 on the right/top faces of c and -1 on its left/bottom faces.

Sides (left, right, bottom, top), each one of:
* "periodic"  -- wrap (both opposite sides);
* "outflow"   -- zero gradient: the outside state is the cell's own nodal state;
* "dirichlet" -- the ghost cell keeps its initial moments; its duals are converged once at the start;
* "slip"      -- wall: the outside state is the cell's state with the momentum reflected about the
                 face, m -> m - 2 (m.n) n (mass flux through the wall vanishes).

Time step (the paper states only "CFL"): dt = CFL * h / s_max, h = min over interior cells of
A_c / (longest face of c), s_max = max over interior and dirichlet ghost cells and all nodes of
max(|v_1|, |v_2|) + c; the last step is clipped to t_end.

Initial data (cell averages at each node; initial duals = projection of the nodal entropy variables,
dirichlet ghosts then converged):
* FreestreamIC: a uniform state rho, p, Mach M(xi), flow angle theta(xi) (degrees):
  v = M sqrt(gamma p / rho) (cos theta, sin theta).
* ShearIC: a horizontal band |y - y_mid| < w(xi) with state (rho_in, v_in) and (rho_out, v_out) outside,
  pressure p, and a transverse velocity v_2 = A(xi) sin(k (x + phase(xi))). The band is averaged
  exactly over the cell's y-extent (fraction f inside); v_2 is taken at the cell centre's x
  (rectangular cells): <rho> = f rho_in + (1-f) rho_out, <rho v_1> = f rho_in v_in + (1-f) rho_out v_out,
  <rho v_2> = <rho> v_2, <E> = p/(gamma-1) + f rho_in (v_in^2 + v_2^2)/2 + (1-f) rho_out (v_out^2 + v_2^2)/2.

Steady residual (Eq. residualSteady, density mean, area-weighted): sum_c A_c |u_{c,0,0}^{n+1} - u_{c,0,0}^n|.

Pinned by: tests/test_oracle_scheme2d.py (geometry closes, constant states and freestream
preserved, conservation on periodic meshes, the deterministic limit against an independent
per-face loop solver with slip walls on the ramp mesh, y-uniform data reproducing the 1-D scheme).
"""
from dataclasses import dataclass, field

import numpy as np

from . import dual as dualmod
from .physics import rusanov


# ------------------------------------------------------------------------------------------------
# meshes
# ------------------------------------------------------------------------------------------------
@dataclass
class Mesh2D:
    X: np.ndarray           # (nx+1, ny+1)
    Y: np.ndarray

    @property
    def nx(self):
        return self.X.shape[0] - 1

    @property
    def ny(self):
        return self.X.shape[1] - 1

    def area(self):
        X, Y = self.X, self.Y
        x0, y0 = X[:-1, :-1], Y[:-1, :-1]
        x1, y1 = X[1:, :-1], Y[1:, :-1]
        x2, y2 = X[1:, 1:], Y[1:, 1:]
        x3, y3 = X[:-1, 1:], Y[:-1, 1:]
        a = 0.5 * ((x0 * y1 - x1 * y0) + (x1 * y2 - x2 * y1) + (x2 * y3 - x3 * y2) + (x3 * y0 - x0 * y3))
        return a.T                                         # (ny, nx)

    def x_faces(self):
        """Unit normals (ny, nx+1, 2) and lengths (ny, nx+1) of the faces between columns."""
        dx = self.X[:, 1:] - self.X[:, :-1]                # along the face, (nx+1, ny)
        dy = self.Y[:, 1:] - self.Y[:, :-1]
        L = np.hypot(dx, dy)
        n = np.stack([dy / L, -dx / L], axis=-1)           # rotate the upward edge by -90 degrees
        return np.transpose(n, (1, 0, 2)), L.T

    def y_faces(self):
        """Unit normals (ny+1, nx, 2) and lengths (ny+1, nx) of the faces between rows."""
        dx = self.X[1:, :] - self.X[:-1, :]                # (nx, ny+1)
        dy = self.Y[1:, :] - self.Y[:-1, :]
        L = np.hypot(dx, dy)
        n = np.stack([-dy / L, dx / L], axis=-1)           # rotate the rightward edge by +90 degrees
        return np.transpose(n, (1, 0, 2)), L.T

    def h_min(self):
        _, lx = self.x_faces()
        _, ly = self.y_faces()
        longest = np.maximum.reduce([lx[:, :-1], lx[:, 1:], ly[:-1, :], ly[1:, :]])
        return float(np.min(self.area() / longest))

    def centres(self):
        xc = 0.25 * (self.X[:-1, :-1] + self.X[1:, :-1] + self.X[1:, 1:] + self.X[:-1, 1:])
        yc = 0.25 * (self.Y[:-1, :-1] + self.Y[1:, :-1] + self.Y[1:, 1:] + self.Y[:-1, 1:])
        return xc.T, yc.T                                  # (ny, nx)


def cartesian_mesh(nx, ny, x_lo, x_hi, y_lo, y_hi) -> Mesh2D:
    x = np.linspace(x_lo, x_hi, nx + 1)
    y = np.linspace(y_lo, y_hi, ny + 1)
    X, Y = np.meshgrid(x, y, indexing="ij")
    return Mesh2D(X, Y)


def ramp_mesh(nx, ny, x_lo, x_hi, y_top, ramp_x0, ramp_deg) -> Mesh2D:
    """Lower wall flat up to ramp_x0, then rising at ramp_deg; upper boundary y = y_top; vertical
    grid lines, rows mapped linearly between the wall and the top: y = y_b(x) + (y_top - y_b(x)) eta."""
    x = x_lo + (x_hi - x_lo) * np.arange(nx + 1) / nx
    eta = np.arange(ny + 1) / ny
    yb = np.where(x > ramp_x0, (x - ramp_x0) * np.tan(np.deg2rad(ramp_deg)), 0.0)
    X = np.repeat(x[:, None], ny + 1, axis=1)
    Y = yb[:, None] + (y_top - yb[:, None]) * eta[None, :]
    return Mesh2D(X, Y)


# ------------------------------------------------------------------------------------------------
# initial data
# ------------------------------------------------------------------------------------------------
def _affine(v0, dv, nodes):
    dv = np.asarray(dv, dtype=np.float64)
    return v0 + nodes @ dv[:nodes.shape[1]]


@dataclass
class FreestreamIC:
    rho: float
    p: float
    mach: float
    angle_deg: float
    dmach: tuple = (0.0, 0.0, 0.0)
    dangle: tuple = (0.0, 0.0, 0.0)

    def cell_states(self, phys, mesh, nodes, ny2, nx2):
        g = phys.gamma
        M = _affine(self.mach, self.dmach, nodes)                 # (Q,)
        th = np.deg2rad(_affine(self.angle_deg, self.dangle, nodes))
        c = np.sqrt(g * self.p / self.rho)
        v1, v2 = M * c * np.cos(th), M * c * np.sin(th)
        u = np.stack([np.full_like(M, self.rho), self.rho * v1, self.rho * v2,
                      self.p / (g - 1.0) + 0.5 * self.rho * (v1 * v1 + v2 * v2)], axis=-1)
        return np.broadcast_to(u, (ny2, nx2) + u.shape).copy()


@dataclass
class RiemannXIC:
    """One jump in x at x0 + dx0 . xi, uniform in y: primitive (rho, v_1, v_2, p) states left and right,
    each affine in xi (rows of d... are the xi-derivatives of the four primitives). Exact cell averages
    in x (rectangular cells), node by node."""
    left: tuple
    right: tuple
    x0: float
    dleft: tuple = ((0.0, 0.0, 0.0),) * 4
    dright: tuple = ((0.0, 0.0, 0.0),) * 4
    dx0: tuple = (0.0, 0.0, 0.0)

    def _state(self, phys, prim0, dprim, nodes):
        g = phys.gamma
        pr = [_affine(prim0[k], dprim[k], nodes) for k in range(4)]
        rho, v1, v2, p = pr
        return np.stack([rho, rho * v1, rho * v2, p / (g - 1.0) + 0.5 * rho * (v1 * v1 + v2 * v2)], axis=-1)

    def cell_states(self, phys, mesh, nodes, ny2, nx2):
        UL = self._state(phys, self.left, self.dleft, nodes)          # (Q, 4)
        UR = self._state(phys, self.right, self.dright, nodes)
        x = mesh.X[:, 0]
        dx = x[1] - x[0]
        xl = np.concatenate([[x[0] - dx], x[:-1], [x[-1]]])           # left edges incl. ghosts
        x0 = _affine(self.x0, self.dx0, nodes)                         # (Q,)
        frac = np.clip((x0[None, :] - xl[:, None]) / dx, 0.0, 1.0)    # (nx+2, Q)
        u = frac[:, :, None] * UL[None] + (1 - frac[:, :, None]) * UR[None]   # (nx+2, Q, 4)
        return np.broadcast_to(u[None], (ny2,) + u.shape).copy()


@dataclass
class ShearIC:
    rho_in: float
    v_in: float
    rho_out: float
    v_out: float
    p: float
    amp: float
    phase: float
    half_width: float
    k: float
    y_mid: float = 0.5
    damp: tuple = (0.0, 0.0, 0.0)
    dphase: tuple = (0.0, 0.0, 0.0)
    dhalf_width: tuple = (0.0, 0.0, 0.0)

    def cell_states(self, phys, mesh, nodes, ny2, nx2):
        """Ghost cells repeat the periodic interior (the update never reads them)."""
        g = phys.gamma
        A = _affine(self.amp, self.damp, nodes)
        ph = _affine(self.phase, self.dphase, nodes)
        w = _affine(self.half_width, self.dhalf_width, nodes)
        ny, nx = mesh.ny, mesh.nx
        xc, _ = mesh.centres()
        ylo = mesh.Y[:-1, :-1].T                          # (ny, nx) rectangular cells
        yhi = mesh.Y[:-1, 1:].T
        lo = self.y_mid - w                               # (Q,)
        hi = self.y_mid + w
        inside = np.clip(np.minimum(yhi[..., None], hi) - np.maximum(ylo[..., None], lo), 0.0, None)
        f = inside / (yhi - ylo)[..., None]               # (ny, nx, Q)
        v2 = A * np.sin(self.k * (xc[..., None] + ph))
        rho = f * self.rho_in + (1 - f) * self.rho_out
        m1 = f * self.rho_in * self.v_in + (1 - f) * self.rho_out * self.v_out
        E = (self.p / (g - 1.0) + 0.5 * f * self.rho_in * (self.v_in ** 2 + v2 ** 2)
             + 0.5 * (1 - f) * self.rho_out * (self.v_out ** 2 + v2 ** 2))
        inner = np.stack([rho, m1, rho * v2, E], axis=-1)         # (ny, nx, Q, 4)
        out = np.empty((ny2, nx2) + inner.shape[2:])
        out[1:-1, 1:-1] = inner
        out[0, 1:-1], out[-1, 1:-1] = inner[-1], inner[0]
        out[:, 0], out[:, -1] = out[:, -2], out[:, 1]
        return out


# ------------------------------------------------------------------------------------------------
# problem and state
# ------------------------------------------------------------------------------------------------
@dataclass
class Problem2D:
    phys: object
    ent: object
    space: object
    mesh: Mesh2D
    ic: object
    sides: tuple = ("periodic", "periodic", "periodic", "periodic")   # left, right, bottom, top
    cfl: float = 0.4
    t_end: float = 0.0
    newton: dualmod.NewtonOptions = field(default_factory=dualmod.NewtonOptions)


@dataclass
class State2D:
    uhat: np.ndarray      # (ny+2, nx+2, N, m)
    lam: np.ndarray
    t: float = 0.0
    n: int = 0
    last_dt: float = 0.0
    newton_iters: np.ndarray = None
    newton_status: np.ndarray = None
    residual: float = np.inf


def _dirichlet_mask(prob: Problem2D):
    ny, nx = prob.mesh.ny, prob.mesh.nx
    m = np.zeros((ny + 2, nx + 2), dtype=bool)
    left, right, bottom, top = prob.sides
    if left == "dirichlet":
        m[1:-1, 0] = True
    if right == "dirichlet":
        m[1:-1, -1] = True
    if bottom == "dirichlet":
        m[0, 1:-1] = True
    if top == "dirichlet":
        m[-1, 1:-1] = True
    return m


def initial_state(prob: Problem2D) -> State2D:
    sp = prob.space
    ny, nx = prob.mesh.ny, prob.mesh.nx
    ubar = prob.ic.cell_states(prob.phys, prob.mesh, sp.nodes, ny + 2, nx + 2)   # (ny+2, nx+2, Q, m)
    uhat = sp.project(ubar)
    lam = sp.project(prob.ent.grad_s(ubar))
    st = State2D(uhat=uhat, lam=lam)
    d = _dirichlet_mask(prob)
    if np.any(d):
        lg, _, stat, _ = dualmod.dual_solve(sp, prob.ent, lam[d], uhat[d], prob.newton)
        assert np.all(stat == 0)
        st.lam[d] = lg
    return st


def nodal_states(prob: Problem2D, lam: np.ndarray) -> np.ndarray:
    return prob.ent.u_s(prob.space.evaluate(lam))


def _reflect(u, n):
    """Momentum reflected about a face with unit normal n (broadcast over nodes)."""
    out = np.array(u, copy=True)
    mn = u[..., 1] * n[..., 0] + u[..., 2] * n[..., 1]
    out[..., 1] = u[..., 1] - 2.0 * mn * n[..., 0]
    out[..., 2] = u[..., 2] - 2.0 * mn * n[..., 1]
    return out


def _outside(prob, side, U, inner, ghost, n):
    """Nodal states beyond a boundary face row/column: inner = the cells next to it, ghost = the
    ghost cells there (ny or nx of them), n = the face normals (any orientation)."""
    if side == "outflow":
        return inner
    if side in ("dirichlet", "periodic"):
        return ghost
    if side == "slip":
        return _reflect(inner, n[..., None, :])
    raise ValueError(side)


def moment_update(prob: Problem2D, lam: np.ndarray, dt: float) -> np.ndarray:
    """c(...) for every interior cell: (ny, nx, N, m)."""
    return prob.space.project(nodal_update(prob, nodal_states(prob, lam), dt))


def nodal_update(prob: Problem2D, U: np.ndarray, dt: float) -> np.ndarray:
    """The finite-volume update of nodal states U (ny+2, nx+2, Q, m), node by node, for every interior
    cell: u_k^(c) - dt/A_c sum_faces L_f s_f g(u_k^(in), u_k^(out); n_f): (ny, nx, Q, m)."""
    mesh = prob.mesh
    left, right, bottom, top = prob.sides
    if left == "periodic":
        U = U.copy()
        U[1:-1, 0], U[1:-1, -1] = U[1:-1, -2], U[1:-1, 1]
    if bottom == "periodic":
        U = U.copy()
        U[0, 1:-1], U[-1, 1:-1] = U[-2, 1:-1], U[1, 1:-1]
    nxf, lxf = mesh.x_faces()                              # (ny, nx+1, 2)
    nyf, lyf = mesh.y_faces()                              # (ny+1, nx, 2)
    C = U[1:-1, 1:-1]                                      # (ny, nx, Q, m)
    # states on both sides of every x-face (behind = lower i, ahead = higher i)
    behind_x = np.concatenate([_outside(prob, left, U, C[:, :1], U[1:-1, :1], nxf[:, :1]), C], axis=1)
    ahead_x = np.concatenate([C, _outside(prob, right, U, C[:, -1:], U[1:-1, -1:], nxf[:, -1:])], axis=1)
    Gx = rusanov(prob.phys, behind_x, ahead_x, nxf[:, :, None, :]) * lxf[:, :, None, None]   # (ny, nx+1, Q, m)
    behind_y = np.concatenate([_outside(prob, bottom, U, C[:1], U[:1, 1:-1], nyf[:1]), C], axis=0)
    ahead_y = np.concatenate([C, _outside(prob, top, U, C[-1:], U[-1:, 1:-1], nyf[-1:])], axis=0)
    Gy = rusanov(prob.phys, behind_y, ahead_y, nyf[:, :, None, :]) * lyf[:, :, None, None]   # (ny+1, nx, Q, m)
    div = (Gx[:, 1:] - Gx[:, :-1]) + (Gy[1:] - Gy[:-1])
    return C - (dt / mesh.area())[..., None, None] * div


def time_step(prob: Problem2D, U: np.ndarray, t: float, clip: bool = True) -> float:
    d = _dirichlet_mask(prob)
    inner = np.zeros(d.shape, dtype=bool)
    inner[1:-1, 1:-1] = True
    smax = float(np.max(prob.phys.speed(U[inner | d])))
    dt = prob.cfl * prob.mesh.h_min() / smax
    if clip and prob.t_end > 0 and t + dt > prob.t_end:
        dt = prob.t_end - t
    return dt


def steady_residual(prob: Problem2D, uhat_new, uhat_old) -> float:
    a = prob.mesh.area()
    return float(np.sum(a * np.abs(uhat_new[1:-1, 1:-1, 0, 0] - uhat_old[1:-1, 1:-1, 0, 0])))


def _solve_interior(prob, st, one_step):
    lam = st.lam.copy()
    li, it, stat, _ = dualmod.dual_solve(prob.space, prob.ent, st.lam[1:-1, 1:-1].reshape(-1, *st.lam.shape[2:]),
                                         st.uhat[1:-1, 1:-1].reshape(-1, *st.uhat.shape[2:]), prob.newton,
                                         one_step=one_step)
    ny, nx = prob.mesh.ny, prob.mesh.nx
    lam[1:-1, 1:-1] = li.reshape(ny, nx, *li.shape[1:])
    return lam, it.reshape(ny, nx), stat.reshape(ny, nx)


def ipm_step(prob: Problem2D, st: State2D) -> State2D:
    """One time step of Algorithm 1 (dual solves in the interior; dirichlet ghosts stay converged)."""
    lam, it, stat = _solve_interior(prob, st, one_step=False)
    U = nodal_states(prob, lam)
    dt = time_step(prob, U, st.t)
    uhat = st.uhat.copy()
    uhat[1:-1, 1:-1] = moment_update(prob, lam, dt)
    return State2D(uhat=uhat, lam=lam, t=st.t + dt, n=st.n + 1, last_dt=dt, newton_iters=it,
                   newton_status=stat, residual=steady_residual(prob, uhat, st.uhat))


def oneshot_step(prob: Problem2D, st: State2D) -> State2D:
    """One pseudo-time step of Algorithm 2 (one damped Newton step per interior cell)."""
    lam, it, stat = _solve_interior(prob, st, one_step=True)
    U = nodal_states(prob, lam)
    dt = time_step(prob, U, st.t, clip=False)
    uhat = st.uhat.copy()
    uhat[1:-1, 1:-1] = moment_update(prob, lam, dt)
    return State2D(uhat=uhat, lam=lam, t=st.t + dt, n=st.n + 1, last_dt=dt, newton_iters=it,
                   newton_status=stat, residual=steady_residual(prob, uhat, st.uhat))
