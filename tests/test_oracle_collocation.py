"""Pins of the Stochastic Collocation oracle (oracle/collocation.py): every node against the
independent plain-loop deterministic solvers of the scheme tests (1-D global Lax-Friedrichs, 2-D
Rusanov on the ramp mesh with a slip wall), conservation node by node, the deterministic limit, the
Burgers expectation against the exact Rankine-Hugoniot solution, steady runs."""
import numpy as np

from oracle import collocation as sc
from oracle import physics
from oracle import scheme1d as s1
from oracle import scheme2d as s2
from tests.test_oracle_scheme import burgers_problem, det_lf, exact_expectation_cell_avgs, rel_l2, sod_problem
from tests.test_oracle_scheme2d import _loop_solver, _problem


def test_every_burgers_node_is_the_plain_lf_solver_with_its_own_time_step():
    prob = burgers_problem(nx=60, M=3, nq=5, t_end=0.05)
    r = sc.run_1d(prob)
    U0 = sc.initial_nodal_1d(prob)
    for k in range(prob.space.Q):
        ref = det_lf(lambda u: 0.5 * u * u, lambda u: abs(u[0]), U0[:, k], prob.dx, prob.cfl, prob.t_end)
        np.testing.assert_allclose(r.U[:, k], ref, rtol=1e-13, atol=1e-13)
        assert r.t[k] == prob.t_end


def test_every_sod_node_is_the_plain_lf_solver():
    prob = sod_problem(nx=40, p=3, M=1, nq=2, t_end=0.05)
    ph = physics.Euler(1.4, 1)
    r = sc.run_1d(prob)
    U0 = sc.initial_nodal_1d(prob)
    for k in range(prob.space.Q):
        ref = det_lf(lambda u: ph.flux(u[None])[0], lambda u: float(ph.speed(u[None])[0]), U0[:, k], prob.dx,
                     prob.cfl, prob.t_end)
        np.testing.assert_allclose(r.U[:, k], ref, rtol=1e-12, atol=1e-12)
    # density and energy vary across the nodes (the uncertain left state), and so do the wave speeds:
    # each node takes its own time steps
    assert np.ptp(r.U[1:-1, :, 0], axis=1).max() > 1e-2
    assert len(set(r.steps.tolist())) > 1 and np.all(r.t == prob.t_end)


def test_every_ramp_node_is_the_plain_face_loop_solver():
    mesh = s2.ramp_mesh(10, 5, 0.0, 2.0, 1.0, 0.5, 15.0)
    ic = s2.FreestreamIC(rho=1.0, p=1.0, mach=2.0, angle_deg=10.0, dmach=(0.1, 0.0, 0.0), dangle=(0.0, 1.0, 0.0))
    prob = _problem(mesh, ic, ("dirichlet", "outflow", "slip", "dirichlet"), p=2, M=1, nq=2)
    r = sc.run_2d(prob, steady_tol=0.0, max_steps=4)
    U0 = sc.initial_nodal_2d(prob)
    assert np.all(r.steps == 4)
    for k in range(prob.space.Q):
        ubar = U0[1, 1, k]
        ref = _loop_solver(mesh.X, mesh.Y, ubar, ubar, 4, prob.cfl)
        assert np.abs(r.U[1:-1, 1:-1, k] - ref).max() < 1e-12 * np.abs(ref).max()
    assert np.ptp(r.U[1:-1, 1:-1, :, 0], axis=-1).max() > 1e-3    # the nodes differ


def test_conservation_node_by_node_on_periodic_meshes():
    prob = burgers_problem(nx=50, M=2, nq=4, t_end=0.03, bc="periodic", x0=lambda xi: 1.5 + 0.3 * xi[:, 0])
    r = sc.run_1d(prob)
    U0 = sc.initial_nodal_1d(prob)
    tot0, tot = U0[1:-1].sum(axis=0), r.U[1:-1].sum(axis=0)
    assert np.abs(tot - tot0).max() < 1e-12 * np.abs(tot0).max()
    assert np.abs(r.U - U0).max() > 1.0                           # the shocks moved

    mesh = s2.cartesian_mesh(10, 10, 0.0, 1.0, 0.0, 1.0)
    ic = s2.ShearIC(rho_in=2.0, v_in=-0.5, rho_out=1.0, v_out=0.5, p=2.5, amp=0.05, phase=0.0, half_width=0.25,
                    k=4 * np.pi, damp=(0.025, 0.0, 0.0), dphase=(0.0, 0.1, 0.0), dhalf_width=(0.0, 0.0, 0.02))
    prob2 = _problem(mesh, ic, ("periodic",) * 4, p=3, M=1, nq=2)
    prob2.t_end = 0.02
    r2 = sc.run_2d(prob2)
    V0 = sc.initial_nodal_2d(prob2)
    A = mesh.area()[..., None, None]
    t0, t1 = np.sum(A * V0[1:-1, 1:-1], axis=(0, 1)), np.sum(A * r2.U[1:-1, 1:-1], axis=(0, 1))
    assert np.abs(t1 - t0).max() < 1e-13 * np.abs(t0).max()
    assert np.all(r2.t == 0.02)


def test_node_independent_data_gives_the_ipm_deterministic_limit():
    prob = burgers_problem(nx=40, M=3, nq=5, x0=lambda xi: np.full(xi.shape[0], 0.5), t_end=0.04)
    r = sc.run_1d(prob)
    m = r.moments(prob.space)
    ipm = s1.run(prob)
    np.testing.assert_allclose(m[:, 0, 0], ipm.uhat[:, 0, 0], rtol=0, atol=1e-8)
    assert np.abs(m[:, 1:]).max() < 1e-12
    assert np.all(r.steps == ipm.n)


def test_burgers_expectation_converges_to_rankine_hugoniot():
    """SC with many nodes: E[u] approaches the exact expectation as the mesh is refined (first-order
    LF); with only 5 nodes the error stalls at the quadrature's aliasing level."""
    errs = {}
    for nx, nq in [(200, 40), (400, 40), (400, 5)]:
        prob = burgers_problem(nx=nx, M=1, nq=nq)
        r = sc.run_1d(prob)
        E = r.moments(prob.space)[:, 0, 0]
        errs[nx, nq] = rel_l2(E[1:-1], exact_expectation_cell_avgs(nx, prob.dx, prob.t_end), prob.dx)
    assert errs[200, 40] < 1.5e-2
    assert errs[400, 40] < 0.75 * errs[200, 40]
    assert errs[400, 5] > 1.5 * errs[400, 40]


def test_steady_ramp_nodes_end_below_the_tolerance():
    mesh = s2.ramp_mesh(8, 4, 0.0, 2.0, 1.0, 0.5, 15.0)
    ic = s2.FreestreamIC(rho=1.0, p=1.0, mach=2.0, angle_deg=10.0, dmach=(0.1, 0.0, 0.0), dangle=(0.0, 1.0, 0.0))
    prob = _problem(mesh, ic, ("dirichlet", "outflow", "slip", "dirichlet"), p=2, M=1, nq=2)
    r = sc.run_2d(prob, steady_tol=1e-8, max_steps=5000)
    assert np.all(r.residual < 1e-8) and np.all(r.steps < 5000)
    # each node's end state is a fixed point of its own scheme
    for k in range(prob.space.Q):
        u = r.U[:, :, k:k + 1]
        dt = s2.time_step(prob, u, 0.0, clip=False)
        assert np.abs(s2.nodal_update(prob, u, dt) - u[1:-1, 1:-1]).max() < 1e-6
