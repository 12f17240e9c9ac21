"""GPU parity of the FP32-factorisation mixed mode (precision "mixed_f32f") against the oracle.

This mode keeps the split-BF16 tensor-core Hessian of the mixed mode and also factorises it, and
solves for the Newton direction, in FP32 on the CUDA cores; the gradient, the stopping test
(Eq. tauCrit), the line search and the update stay in FP64. The Newton direction is then exact to
about cond(H) * 2^-24 relative on top of the Hessian's own ~2^-15, so Newton still converges
(linearly with a tiny rate near the solution) to a point that meets the FP64 stopping test; the
results are held to the mixed-mode tolerance 1e-6 and the count of Newton updates to a small excess
over the oracle's. A non-positive FP32 pivot sends the cell through the FP64 factorisation instead
(counted in fp32_fallbacks)."""
import numpy as np
import pytest

from oracle import dual
from oracle import scheme1d as s1
from oracle import scheme2d as s2
from paper_1912_09238_gb300 import ipm, workloads
from tests._cases import gpu_context, oracle_problem, oracle_problem_2d, rel_err

pytestmark = pytest.mark.gpu
TOL_MIXED = 1e-6
PREC = "mixed_f32f"

SOD_SMALL = workloads.variant(workloads.SOD_1D, nx=64, t_end=0.14)


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_09238_gb300 import build
    build.build()


@pytest.mark.parametrize("w", [
    workloads.BURGERS_1D,
    SOD_SMALL,
    # N = 120, m = 3: H in HBM, two passes through tensor memory
    workloads.variant(workloads.SOD_1D, nx=3, M=7, nq=8, x_lo=0.49, x_hi=0.51),
], ids=["burgers", "sod", "sod_deg7"])
def test_dual_solve_from_initial_data(w):
    prob = oracle_problem(w)
    st = s1.initial_state(prob)
    lam, it, stat, _ = dual.dual_solve(prob.space, prob.ent, st.lam[1:-1], st.uhat[1:-1], prob.newton)
    assert np.all(stat == 0)
    ctx = gpu_context(w, precision=PREC)
    s = ctx.dual_solve()
    assert s.failed_cells == 0 and s.tc_timeouts == 0 and s.fp32_fallbacks == 0
    g = ctx.get_duals()[1:-1]
    assert rel_err(g, lam) < TOL_MIXED
    U = prob.ent.u_s(prob.space.evaluate(lam))
    assert rel_err(np.swapaxes(ctx.get_nodal_states()[1:-1], 1, 2), U) < TOL_MIXED
    assert s.newton_iters <= int(1.5 * it.sum()) + 2
    assert s.factorizations == s.newton_iters
    ctx.close()


def test_sod_steps_match_oracle():
    prob = oracle_problem(SOD_SMALL)
    st = s1.initial_state(prob)
    ctx = gpu_context(SOD_SMALL, precision=PREC)
    for n in range(12):
        st = s1.ipm_step(prob, st)
        s = ctx.step()
        assert s.failed_cells == 0 and s.tc_timeouts == 0
        assert abs(s.dt - st.last_dt) <= 1e-6 * st.last_dt
        assert rel_err(ctx.get_moments(), st.uhat) < TOL_MIXED, n
    assert ctx.sync_stats().fp32_fallbacks == 0
    ctx.close()


def test_burgers_full_run():
    prob = oracle_problem(workloads.BURGERS_1D)
    ref = s1.run(prob)
    ctx = gpu_context(workloads.BURGERS_1D, precision=PREC)
    s = ctx.run()
    assert s.failed_cells == 0 and s.tc_timeouts == 0
    assert s.steps == ref.n
    assert rel_err(ctx.get_moments(), ref.uhat) < TOL_MIXED
    ctx.close()


def test_ramp_oneshot_cta_kernel():
    """N m = 60 would take the warp-per-cell kernel in the other modes; this mode always runs the
    CTA-per-cell kernel (tensor-core Hessian)."""
    w = workloads.variant(workloads.RAMP_2D, nx=12, ny=6, M=4, nq=5)
    prob = oracle_problem_2d(w)
    st = s2.initial_state(prob)
    ctx = gpu_context(w, precision=PREC)
    assert ctx.tuning()[0] == 1
    for _ in range(6):
        st = s2.oneshot_step(prob, st)
        assert ctx.oneshot_step().failed_cells == 0
    got = ctx.get_moments().reshape(st.uhat.shape)[1:-1, 1:-1]
    assert rel_err(got, st.uhat[1:-1, 1:-1]) < TOL_MIXED
    ctx.close()


def test_sod_full_size_first_step_sampled():
    w = workloads.SOD_1D
    prob = oracle_problem(w)
    st = s1.initial_state(prob)
    ctx = gpu_context(w, precision=PREC)
    s = ctx.step()
    assert s.failed_cells == 0 and s.tc_timeouts == 0 and s.fp32_fallbacks == 0
    got = ctx.get_moments()
    flat = np.concatenate([st.uhat.reshape(st.uhat.shape[0], -1), st.lam.reshape(st.lam.shape[0], -1)], axis=1)
    _, first, inverse = np.unique(flat, axis=0, return_index=True, return_inverse=True)
    lu, _, stat, _ = dual.dual_solve(prob.space, prob.ent, st.lam[first], st.uhat[first], prob.newton)
    assert np.all(stat == 0)
    lam = lu[inverse.reshape(-1)]
    U = s1.nodal_states(prob, lam)
    dt = s1.time_step(prob, U, 0.0)
    assert abs(s.dt - dt) <= 1e-9 * dt
    sample = np.unique(np.r_[1, 2, 999, 1000, 1001, 1002, 2000, np.random.default_rng(5).integers(1, 2001, 12)])
    full = s1.moment_update(prob, lam, dt)
    assert rel_err(got[sample], full[sample - 1]) < TOL_MIXED
    ctx.close()


def test_rejects_frozen_hessians():
    with pytest.raises(ipm.IpmError):
        gpu_context(SOD_SMALL, precision=PREC, hessian_reuse=1)


def test_adaptive_shear_layer_matches_the_oracle():
    """Adaptive degrees 2-4 on the shear layer: the degree-2 cells on the warp kernel (FP64
    factorisation of their small systems), the others with the FP32 factorisation."""
    from oracle import adaptive as ad
    w = workloads.variant(workloads.KH_2D, nx=12, ny=12, M=4, nq=5)
    lv = ad.Levels(degrees=(2, 3, 4), delta_lo=2e-4, delta_hi=2e-5)
    prob = oracle_problem_2d(w)
    st = ad.initial_state(prob, lv)
    ctx = gpu_context(w, precision=PREC, adapt_min_degree=2, delta_lo=2e-4, delta_hi=2e-5)
    for n in range(4):
        st = ad.ipm_step(prob, st, lv)
        s = ctx.step()
        assert s.failed_cells == 0 and s.tc_timeouts == 0
        lev = ctx.get_levels().reshape(st.level.shape)
        assert np.array_equal(lev[1:-1, 1:-1], st.level[1:-1, 1:-1]), n
        got = ctx.get_moments().reshape(st.uhat.shape)
        assert rel_err(got[1:-1, 1:-1], st.uhat[1:-1, 1:-1]) < TOL_MIXED, n
    ctx.close()
