"""GPU parity of the FP64 path against the oracle, through the C ABI (1-D problems).

Tolerance: 1e-10 normwise relative (max|gpu - oracle| / max|oracle|) for FP64 results. Inputs are
the workloads' own initial data (each side projects it itself) or oracle-made states."""
import numpy as np
import pytest

from oracle import dual
from oracle import scheme1d as s1
from paper_1912_09238_gb300 import workloads
from tests._cases import gpu_context, oracle_problem, rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-10

BURGERS = workloads.BURGERS_1D
SOD_SMALL = workloads.variant(workloads.SOD_1D, nx=64, t_end=0.14)
SOD_LOW = workloads.variant(workloads.SOD_1D, nx=50, M=2, nq=3)


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_09238_gb300 import build
    build.build()


@pytest.mark.parametrize("w", [BURGERS, SOD_SMALL, SOD_LOW], ids=["burgers", "sod", "sod_low"])
def test_initial_data_projection(w):
    prob = oracle_problem(w)
    st = s1.initial_state(prob)
    ctx = gpu_context(w)
    assert rel_err(ctx.get_moments(), st.uhat) < 1e-13
    assert rel_err(ctx.get_duals(), st.lam) < 1e-12


@pytest.mark.parametrize("w", [BURGERS, SOD_SMALL, SOD_LOW], ids=["burgers", "sod", "sod_low"])
def test_dual_solve_from_initial_data(w):
    prob = oracle_problem(w)
    st = s1.initial_state(prob)
    lam, it, stat, _ = dual.dual_solve(prob.space, prob.ent, st.lam[1:-1], st.uhat[1:-1], prob.newton)
    assert np.all(stat == 0)
    ctx = gpu_context(w)
    s = ctx.dual_solve()
    assert s.failed_cells == 0
    g = ctx.get_duals()[1:-1]
    assert rel_err(g, lam) < TOL
    assert s.newton_iters == int(it.sum())
    # nodal states the update will use are u_s at the solved duals
    U = prob.ent.u_s(prob.space.evaluate(lam))                      # (C, Q, m)
    assert rel_err(np.swapaxes(ctx.get_nodal_states()[1:-1], 1, 2), U) < TOL


def test_manufactured_round_trip_sod_full_degree(rng):
    """u_hat = h(lambda*) made by the oracle; the GPU recovers lambda* from a mean-only start."""
    w = workloads.variant(workloads.SOD_1D, nx=40)
    prob = oracle_problem(w, tau=1e-12)
    st = s1.initial_state(prob)
    lam_star = st.lam.copy()
    # perturb the density and momentum duals only: any value there is admissible, while the
    # energy dual Lambda_E must stay negative at every node
    lam_star[:, 1:, :2] += workloads.random_dual_perturbation(lam_star[:, 1:, :2].shape, 7, 0.002)
    assert np.all(prob.ent.feasible(prob.space.evaluate(lam_star)))
    uhat = dual.moments_from_duals(prob.space, prob.ent, lam_star)
    lam0 = np.zeros_like(lam_star)
    lam0[:, 0, :] = lam_star[:, 0, :]
    ref, it, stat, _ = dual.dual_solve(prob.space, prob.ent, lam0[1:-1], uhat[1:-1], prob.newton)
    assert np.all(stat == 0)
    ctx = gpu_context(w, tau=1e-12)
    ctx.set_moments(uhat)
    ctx.set_duals(lam0)
    s = ctx.dual_solve()
    assert s.failed_cells == 0
    g = ctx.get_duals()[1:-1]
    assert rel_err(g, ref) < TOL
    assert rel_err(g, lam_star[1:-1]) < 1e-9
    back = prob.space.project(np.swapaxes(ctx.get_nodal_states()[1:-1], 1, 2))
    assert rel_err(back, uhat[1:-1]) < 1e-12


@pytest.mark.parametrize("w", [BURGERS, SOD_SMALL], ids=["burgers", "sod"])
def test_moment_update_alone(w):
    """Kernel (d) alone: the oracle's converged duals go in, c(...) with a fixed dt comes out."""
    prob = oracle_problem(w)
    st = s1.initial_state(prob)
    lam, _, stat, _ = dual.dual_solve(prob.space, prob.ent, st.lam, st.uhat, prob.newton)
    dt = 0.3 * prob.dx
    ref = s1.moment_update(prob, lam, dt)
    ctx = gpu_context(w)
    ctx.set_duals(lam)
    ctx.set_moments(st.uhat)
    ctx.dual_solve()              # already converged: 0 iterations, nodal states at these duals
    ctx.update(dt)
    assert rel_err(ctx.get_moments()[1:-1], ref) < TOL


def test_burgers_full_run():
    """The Burgers workload end to end (Algorithm 1 to t_end) on both sides."""
    prob = oracle_problem(BURGERS)
    ref = s1.run(prob)
    ctx = gpu_context(BURGERS)
    s = ctx.run()
    assert s.failed_cells == 0
    assert s.steps == ref.n
    assert abs(s.t - ref.t) < 1e-14
    assert rel_err(ctx.get_moments(), ref.uhat) < TOL


def test_sod_steps_match_step_by_step():
    prob = oracle_problem(SOD_SMALL)
    st = s1.initial_state(prob)
    ctx = gpu_context(SOD_SMALL)
    for n in range(12):
        st = s1.ipm_step(prob, st)
        s = ctx.step()
        assert s.failed_cells == 0
        assert abs(s.dt - st.last_dt) <= 1e-12 * st.last_dt
        assert rel_err(ctx.get_moments(), st.uhat) < TOL, n


def test_sod_full_size_first_step_sampled():
    """The 2000-cell Sod workload: the GPU's first step against the oracle on sampled cells
    (each sampled cell needs only its own and its neighbours' dual solves)."""
    w = workloads.SOD_1D
    prob = oracle_problem(w)
    st = s1.initial_state(prob)
    ctx = gpu_context(w)
    s = ctx.step()
    assert s.failed_cells == 0
    got = ctx.get_moments()
    # dt needs the max speed over all cells: the oracle solves each distinct initial cell state once
    # (away from the interface the cells repeat the left or right state exactly)
    flat = np.concatenate([st.uhat.reshape(st.uhat.shape[0], -1), st.lam.reshape(st.lam.shape[0], -1)], axis=1)
    _, first, inverse = np.unique(flat, axis=0, return_index=True, return_inverse=True)
    lu, _, stat, _ = dual.dual_solve(prob.space, prob.ent, st.lam[first], st.uhat[first], prob.newton)
    assert np.all(stat == 0)
    lam = lu[inverse.reshape(-1)]
    U = s1.nodal_states(prob, lam)
    dt = s1.time_step(prob, U, 0.0)
    assert abs(s.dt - dt) <= 1e-12 * dt
    sample = np.unique(np.r_[1, 2, 999, 1000, 1001, 1002, 2000, np.random.default_rng(3).integers(1, 2001, 12)])
    full = s1.moment_update(prob, lam, dt)
    assert rel_err(got[sample], full[sample - 1]) < TOL


@pytest.mark.parametrize("bc", [("periodic", "periodic"), ("dirichlet", "dirichlet"), ("dirichlet", "outflow")])
def test_boundary_conditions(bc):
    w = workloads.variant(BURGERS, nx=37, bc=bc, t_end=0.02)
    prob = oracle_problem(w)
    ref = s1.run(prob)
    ctx = gpu_context(w)
    s = ctx.run()
    assert s.failed_cells == 0 and s.steps == ref.n
    assert rel_err(ctx.get_moments(), ref.uhat) < TOL


def test_quadratic_entropy_is_one_newton_step():
    w = workloads.variant(BURGERS, nx=30, entropy="quadratic", t_end=0.01)
    prob = oracle_problem(w)
    ref = s1.run(prob)
    ctx = gpu_context(w)
    s = ctx.run()
    assert s.max_iters <= 1
    assert rel_err(ctx.get_moments(), ref.uhat) < TOL


@pytest.mark.parametrize("M,nq", [(0, 1), (1, 2), (9, 13)])
def test_degenerate_and_ragged_sizes(M, nq):
    w = workloads.variant(BURGERS, nx=1, M=M, nq=nq, t_end=0.003, x_lo=0.49, x_hi=0.51)
    prob = oracle_problem(w)
    ref = s1.run(prob)
    ctx = gpu_context(w)
    s = ctx.run()
    assert s.failed_cells == 0 and s.steps == ref.n
    assert rel_err(ctx.get_moments(), ref.uhat) < TOL


def test_hessian_in_global_workspace():
    """N*m = 252 (total degree 6, 3 dims, 1-D Euler): the packed Hessian exceeds shared memory and
    lives in the per-CTA global workspace."""
    w = workloads.variant(workloads.SOD_1D, nx=6, M=6, nq=7, t_end=0.0)
    prob = oracle_problem(w)
    st = s1.initial_state(prob)
    ctx = gpu_context(w)
    for _ in range(2):
        st = s1.ipm_step(prob, st)
        s = ctx.step()
        assert s.failed_cells == 0
    assert rel_err(ctx.get_moments(), st.uhat) < TOL


def test_oneshot_matches_oracle():
    w = workloads.variant(BURGERS, nx=30, M=4, nq=8, x_lo=0.0, x_hi=1.0, bc=("dirichlet", "outflow"),
                          u_minus=0.5, u_plus=4.0, t_end=0.0, x0=0.4, dx0=(0.1, 0, 0),
                          left=(2.0,), dleft=((0.5, 0, 0),), right=(3.0,), dright=((0.3, 0, 0),))
    prob = oracle_problem(w)
    st = s1.initial_state(prob)
    ctx = gpu_context(w)
    for n in range(40):
        st = s1.oneshot_step(prob, st)
        s = ctx.oneshot_step()
        assert s.failed_cells == 0
        assert abs(s.residual - st.residual) <= 1e-9 * max(st.residual, 1e-300) + 1e-15
    assert rel_err(ctx.get_moments(), st.uhat) < TOL
    assert rel_err(ctx.get_duals()[1:-1], st.lam[1:-1]) < TOL


def test_infeasible_duals_are_reported_not_fatal():
    w = workloads.variant(workloads.SOD_1D, nx=8, M=2, nq=3)
    ctx = gpu_context(w)
    lam = ctx.get_duals()
    lam[3, 0, 2] = abs(lam[3, 0, 2]) * 10 + 5.0          # Lambda_E > 0 at every node of cell 3
    ctx.set_duals(lam)
    s = ctx.dual_solve()
    assert s.failed_cells == 1 and s.first_failed_cell == 3 and s.first_status == 5
    # the other cells are still solved
    ctx2 = gpu_context(w)
    s2 = ctx2.dual_solve()
    assert s2.failed_cells == 0
