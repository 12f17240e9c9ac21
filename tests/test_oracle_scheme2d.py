"""Pins of the 2-D oracle scheme (oracle/scheme2d.py) against geometry, conservation, an
independent per-face loop solver and the 1-D scheme."""
import numpy as np
import pytest

from oracle import basis, dual, entropy, physics
from oracle import scheme1d as s1
from oracle import scheme2d as s2

GAMMA = 1.4


def _problem(mesh, ic, sides, p=1, M=2, nq=3, cfl=0.4, tau=1e-10):
    sp = basis.StochasticSpace(p, M, nq)
    return s2.Problem2D(phys=physics.Euler(GAMMA, 2), ent=entropy.Euler(GAMMA, 2), space=sp, mesh=mesh, ic=ic,
                        sides=sides, cfl=cfl, newton=dual.NewtonOptions(tau=tau))


def test_ramp_mesh_geometry():
    m = s2.ramp_mesh(16, 8, 0.0, 2.0, 1.0, 0.5, 15.0)
    # total area = channel minus the triangle under the ramp
    assert abs(m.area().sum() - (2.0 - 0.5 * 1.5 * 1.5 * np.tan(np.deg2rad(15.0)))) < 1e-13
    nxf, lxf = m.x_faces()
    nyf, lyf = m.y_faces()
    assert np.allclose(np.linalg.norm(nxf, axis=-1), 1.0) and np.allclose(np.linalg.norm(nyf, axis=-1), 1.0)
    # every cell is closed: sum of outward L n vanishes
    net = (nxf[:, 1:] * lxf[:, 1:, None] - nxf[:, :-1] * lxf[:, :-1, None]
           + nyf[1:] * lyf[1:, :, None] - nyf[:-1] * lyf[:-1, :, None])
    assert np.abs(net).max() < 1e-14
    # the wall normal on the ramp is tilted by 15 degrees
    wall = nyf[0]
    assert np.allclose(wall[0], [0.0, 1.0])
    assert np.allclose(wall[-1], [-np.sin(np.deg2rad(15)), np.cos(np.deg2rad(15))])
    # Cartesian: h = min(dx, dy)
    assert abs(s2.cartesian_mesh(10, 5, 0, 1, 0, 1).h_min() - 0.1) < 1e-15


def test_uncertain_freestream_preserved_on_the_ramp_mesh():
    """A uniform state (any xi) is a steady solution where no wall turns it: only closed cells matter."""
    mesh = s2.ramp_mesh(12, 6, 0.0, 2.0, 1.0, 0.5, 15.0)
    ic = s2.FreestreamIC(rho=1.0, p=1.0, mach=2.0, angle_deg=10.0, dmach=(0.1, 0.0, 0.0), dangle=(0.0, 1.0, 0.0))
    prob = _problem(mesh, ic, ("dirichlet", "outflow", "dirichlet", "dirichlet"), p=2, M=2, nq=3)
    st = s2.initial_state(prob)
    u0 = st.uhat.copy()
    for _ in range(3):
        st = s2.ipm_step(prob, st)
    assert np.abs(st.uhat[1:-1, 1:-1] - u0[1:-1, 1:-1]).max() < 1e-9 * np.abs(u0).max()


def test_conservation_on_a_periodic_mesh():
    mesh = s2.cartesian_mesh(12, 12, 0.0, 1.0, 0.0, 1.0)
    ic = s2.ShearIC(rho_in=2.0, v_in=-0.5, rho_out=1.0, v_out=0.5, p=2.5, amp=0.05, phase=0.0, half_width=0.25,
                    k=4 * np.pi, damp=(0.025, 0.0, 0.0), dphase=(0.0, 0.1, 0.0), dhalf_width=(0.0, 0.0, 0.02))
    prob = _problem(mesh, ic, ("periodic",) * 4, p=3, M=1, nq=2)
    st = s2.initial_state(prob)
    A = mesh.area()[..., None, None]
    for _ in range(3):
        old = st
        lam, _, stat = s2._solve_interior(prob, old, one_step=False)
        assert np.all(stat == 0)
        st = s2.ipm_step(prob, old)
        # fluxes telescope: total of the new moments = total of <u_s(lambda) phi>, to round-off
        proj = prob.space.project(s2.nodal_states(prob, lam))[1:-1, 1:-1]
        tot_new = np.sum(A * st.uhat[1:-1, 1:-1], axis=(0, 1))
        assert np.abs(tot_new - np.sum(A * proj, axis=(0, 1))).max() < 1e-13
        # and the moments move by at most the dual residual of each cell
        drift = np.abs(tot_new - np.sum(A * old.uhat[1:-1, 1:-1], axis=(0, 1))).max()
        assert drift <= mesh.area().sum() * 1e-10


# ------------------------------------------------------------------------------------------------
# an independent deterministic 2-D Euler solver: loops over cells and faces
# ------------------------------------------------------------------------------------------------
def _prim_flux(u, nx_, ny_):
    rho, m1, m2, E = u
    v1, v2 = m1 / rho, m2 / rho
    p = (GAMMA - 1) * (E - 0.5 * rho * (v1 * v1 + v2 * v2))
    vn = v1 * nx_ + v2 * ny_
    f = np.array([rho * vn, m1 * vn + p * nx_, m2 * vn + p * ny_, (E + p) * vn])
    return f, abs(vn) + np.sqrt(GAMMA * p / rho), p


def _loop_solver(X, Y, u_init, u_inflow, steps, cfl):
    """Cells (i, j) with counter-clockwise corners; left/top: inflow state; right: copy; bottom: wall."""
    nx, ny = X.shape[0] - 1, X.shape[1] - 1
    u = {(i, j): u_init.copy() for i in range(nx) for j in range(ny)}
    corners = lambda i, j: [(X[i, j], Y[i, j]), (X[i + 1, j], Y[i + 1, j]), (X[i + 1, j + 1], Y[i + 1, j + 1]),
                            (X[i, j + 1], Y[i, j + 1])]
    geo = {}
    hmin = np.inf
    for i in range(nx):
        for j in range(ny):
            c = corners(i, j)
            area = 0.5 * sum(c[k][0] * c[(k + 1) % 4][1] - c[(k + 1) % 4][0] * c[k][1] for k in range(4))
            faces = []
            for k, nb in enumerate([(i, j - 1), (i + 1, j), (i, j + 1), (i - 1, j)]):     # bottom right top left
                (xa, ya), (xb, yb) = c[k], c[(k + 1) % 4]
                L = np.hypot(xb - xa, yb - ya)
                faces.append((nb, (yb - ya) / L, -(xb - xa) / L, L))                     # outward normal
            geo[i, j] = (area, faces)
            hmin = min(hmin, area / max(f[3] for f in faces))
    smax_in = max(abs(u_inflow[1] / u_inflow[0]), abs(u_inflow[2] / u_inflow[0])) + np.sqrt(
        GAMMA * _prim_flux(u_inflow, 1.0, 0.0)[2] / u_inflow[0])
    for _ in range(steps):
        smax = smax_in
        for v in u.values():
            rho = v[0]
            p = _prim_flux(v, 1.0, 0.0)[2]
            smax = max(smax, max(abs(v[1] / rho), abs(v[2] / rho)) + np.sqrt(GAMMA * p / rho))
        dt = cfl * hmin / smax
        new = {}
        for (i, j), v in u.items():
            area, faces = geo[i, j]
            acc = np.zeros(4)
            for (ni, nj), nx_, ny_, L in faces:
                if 0 <= ni < nx and 0 <= nj < ny:
                    w = u[ni, nj]
                elif ni < 0 or nj >= ny:
                    w = u_inflow
                elif ni >= nx:
                    w = v
                else:                                         # bottom wall: reflect the momentum
                    mn = v[1] * nx_ + v[2] * ny_
                    w = np.array([v[0], v[1] - 2 * mn * nx_, v[2] - 2 * mn * ny_, v[3]])
                fa, sa, _ = _prim_flux(v, nx_, ny_)
                fb, sb, _ = _prim_flux(w, nx_, ny_)
                acc += L * (0.5 * (fa + fb) - 0.5 * max(sa, sb) * (w - v))
            new[i, j] = v - dt / area * acc
        u = new
    out = np.empty((ny, nx, 4))
    for (i, j), v in u.items():
        out[j, i] = v
    return out


def test_deterministic_limit_on_the_ramp_with_a_slip_wall():
    """xi-independent data: IPM's mean equals the deterministic finite-volume scheme, including the
    inflow, far-field, outflow and slip-wall sides on the mapped mesh."""
    mesh = s2.ramp_mesh(10, 5, 0.0, 2.0, 1.0, 0.5, 15.0)
    ic = s2.FreestreamIC(rho=1.0, p=1.0, mach=2.0, angle_deg=10.0)
    prob = _problem(mesh, ic, ("dirichlet", "outflow", "slip", "dirichlet"), p=1, M=2, nq=3)
    st = s2.initial_state(prob)
    for _ in range(4):
        st = s2.ipm_step(prob, st)
        assert np.all(st.newton_status == 0)
    ubar = ic.cell_states(prob.phys, mesh, prob.space.nodes, 1, 1)[0, 0, 0]
    ref = _loop_solver(mesh.X, mesh.Y, ubar, ubar, 4, prob.cfl)
    mean = st.uhat[1:-1, 1:-1, 0, :]                          # phi_0 = 1: the zero-order moment is the mean
    assert np.abs(mean - ref).max() < 1e-8 * np.abs(ref).max()
    assert np.abs(st.uhat[1:-1, 1:-1, 1:, :]).max() < 1e-9    # no xi-dependence appears
    assert np.abs(mean - ubar).max() > 1e-3                   # the wall did turn the flow


def test_x_riemann_problem_reduces_to_the_1d_scheme():
    """Data varying in x only, v_2 = 0, periodic in y: the 2-D scheme (4 variables) equals the 1-D
    scheme with the same (local LF) flux, and the y-momentum and its dual stay zero."""
    nx = 30
    mesh = s2.cartesian_mesh(nx, 2, 0.0, 1.0, 0.0, 0.2)
    left, right = (1.0, 0.0, 0.0, 1.0), (0.125, 0.0, 0.0, 0.1)
    dleft = ((0.1, 0.0, 0.0), (0.0, 0.0, 0.0), (0.0, 0.0, 0.0), (0.0, 0.1, 0.0))
    ic = s2.RiemannXIC(left=left, right=right, x0=0.5, dleft=dleft)
    prob2 = _problem(mesh, ic, ("outflow", "outflow", "periodic", "periodic"), p=2, M=2, nq=3, cfl=0.4)
    sp = prob2.space
    E1 = entropy.Euler(GAMMA, 1)

    def state(prim, d):
        def f(xi):
            pr = [prim[k] + xi @ np.asarray(d[k])[:xi.shape[1]] for k in (0, 1, 3)]
            return E1.conserved(pr[0], pr[1][:, None], pr[2])
        return f
    prob1 = s1.Problem1D(phys=physics.Euler(GAMMA, 1), ent=E1, space=sp, nx=nx, x_lo=0.0, x_hi=1.0,
                         ic=s1.RiemannIC(state(left, dleft), state(right, ((0, 0, 0),) * 4), lambda xi: np.full(len(xi), 0.5)),
                         bc="outflow", cfl=0.4, flux="rusanov")
    prob1.newton = dual.NewtonOptions(tau=1e-10)
    st2 = s2.initial_state(prob2)
    st1 = s1.initial_state(prob1)
    for _ in range(5):
        st2 = s2.ipm_step(prob2, st2)
        st1 = s1.ipm_step(prob1, st1)
        assert abs(st2.last_dt - st1.last_dt) <= 1e-12 * st1.last_dt
    for row in (1, 2):
        u2 = st2.uhat[row, 1:-1]
        assert np.abs(u2[..., [0, 1, 3]] - st1.uhat[1:-1]).max() < 1e-9 * np.abs(st1.uhat).max()
        assert np.abs(u2[..., 2]).max() < 1e-12
        assert np.abs(st2.lam[row, 1:-1, :, 2]).max() < 1e-10


def test_x_riemann_with_uncertain_interface_reduces_to_the_1d_scheme():
    """The Sod data of the 1-D workload in 3 uncertain dims (rho_L, p_L and the interface x0 = 0.5 +
    0.05 xi_3) on a one-row mesh, periodic in y, as the 4-variable 2-D system: it equals the 1-D scheme with
    the same data and flux (the per-node cell averages take the node's interface position on both sides),
    and the y-momentum stays zero. A dropped interface term would leave the xi_3-moments zero."""
    nx = 24
    mesh = s2.cartesian_mesh(nx, 1, 0.0, 1.0, 0.0, 1.0 / nx)
    left, right = (1.0, 0.0, 0.0, 1.0), (0.125, 0.0, 0.0, 0.1)
    dleft = ((0.1, 0.0, 0.0), (0.0, 0.0, 0.0), (0.0, 0.0, 0.0), (0.0, 0.1, 0.0))
    ic = s2.RiemannXIC(left=left, right=right, x0=0.5, dleft=dleft, dx0=(0.0, 0.0, 0.05))
    prob2 = _problem(mesh, ic, ("outflow", "outflow", "periodic", "periodic"), p=3, M=2, nq=3, cfl=0.5)
    sp = prob2.space
    E1 = entropy.Euler(GAMMA, 1)

    def state(prim, d):
        def f(xi):
            pr = [prim[k] + xi @ np.asarray(d[k])[:xi.shape[1]] for k in (0, 1, 3)]
            return E1.conserved(pr[0], pr[1][:, None], pr[2])
        return f
    prob1 = s1.Problem1D(phys=physics.Euler(GAMMA, 1), ent=E1, space=sp, nx=nx, x_lo=0.0, x_hi=1.0,
                         ic=s1.RiemannIC(state(left, dleft), state(right, ((0, 0, 0),) * 4),
                                         lambda xi: 0.5 + 0.05 * xi[:, 2]),
                         bc="outflow", cfl=0.5, flux="rusanov")
    prob1.newton = dual.NewtonOptions(tau=1e-10)
    st2 = s2.initial_state(prob2)
    st1 = s1.initial_state(prob1)
    # the interface moves with xi_3: the first-order xi_3 moment of the density is nonzero at the jump
    i3 = [k for k, a in enumerate(sp.indices) if tuple(a) == (0, 0, 1)][0]
    assert np.abs(st2.uhat[1, 1:-1, i3, 0]).max() > 1e-3
    for _ in range(4):
        st2 = s2.ipm_step(prob2, st2)
        st1 = s1.ipm_step(prob1, st1)
        assert abs(st2.last_dt - st1.last_dt) <= 1e-12 * st1.last_dt
    u2 = st2.uhat[1, 1:-1]
    assert np.abs(u2[..., [0, 1, 3]] - st1.uhat[1:-1]).max() < 1e-9 * np.abs(st1.uhat).max()
    assert np.abs(u2[..., 2]).max() < 1e-12


def test_oneshot_2d_residual_decreases_to_the_steady_ramp_flow():
    """Algorithm 2 on a coarse ramp mesh: the steady residual falls by orders of magnitude."""
    mesh = s2.ramp_mesh(8, 4, 0.0, 2.0, 1.0, 0.5, 15.0)
    ic = s2.FreestreamIC(rho=1.0, p=1.0, mach=2.0, angle_deg=10.0, dmach=(0.1, 0.0, 0.0))
    prob = _problem(mesh, ic, ("dirichlet", "outflow", "slip", "dirichlet"), p=1, M=2, nq=3, cfl=0.4)
    st = s2.initial_state(prob)
    res = []
    for _ in range(400):
        st = s2.oneshot_step(prob, st)
        res.append(st.residual)
    assert res[-1] < 1e-5 * max(res[:5])
    # the One-Shot fixed point is the IPM steady state: converged duals, an Algorithm-1 step leaves it
    lam, _, stat = s2._solve_interior(prob, st, one_step=False)
    assert np.all(stat == 0)
    assert np.abs(lam - st.lam).max() < 1e-6
    nxt = s2.ipm_step(prob, st)
    assert nxt.residual < 2 * res[-1] + 1e-12
