"""GPU parity of the mixed-precision path (tensor-core Hessian) against the oracle, through the C ABI.

The mixed path changes only the Hessian contraction (split-BF16 products, FP32 accumulation on the
tensor cores). Its checks:
* the Hessian itself, element by element, against the oracle's FP64 Hessian within the error bound
  of the split products: |H_mixed - H| <= 2^-12 * sum_k w_k |J_k,ab| |phi_i(xi_k)| |phi_j(xi_k)|
  (each BF16 pair represents its factor to 2^-16 relative, the dropped lo*lo term is 2^-16, the
  FP32 products and sums add a few 2^-24; 2^-12 leaves a factor of ~8 of room);
* everything the path returns (duals, moments, nodal states) against the oracle at 1e-6 relative,
  the mixed-mode tolerance; the gradient and the stopping test stay in FP64, so in practice the
  results agree far more closely, which the tests also record.
The FP64 Hessian of the same entry point is held to 1e-12.
"""
import numpy as np
import pytest

from oracle import dual
from oracle import scheme1d as s1
from paper_1912_09238_gb300 import workloads
from tests._cases import gpu_context, oracle_problem, rel_err

pytestmark = pytest.mark.gpu
TOL_MIXED = 1e-6

BURGERS = workloads.BURGERS_1D
SOD_SMALL = workloads.variant(workloads.SOD_1D, nx=64, t_end=0.14)


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_09238_gb300 import build
    build.build()


def _packed(H):
    r, c = np.tril_indices(H.shape[-1])
    return H[:, r, c]


def _abs_terms(prob, lam):
    """sum_k w_k |J_k,ab| |phi_i| |phi_j| in the flat (i*m + a, j*m + b) layout, packed."""
    sp, ent = prob.space, prob.ent
    J = np.abs(ent.du_s(sp.evaluate(lam)))
    A = np.abs(sp.Phi)
    C, N, m = lam.shape
    T = np.einsum("k,ckab,ki,kj->ciajb", sp.w, J, A, A, optimize=True).reshape(C, N * m, N * m)
    return _packed(T)


def _state_after(prob, steps):
    st = s1.initial_state(prob)
    for _ in range(steps):
        st = s1.ipm_step(prob, st)
    return st


@pytest.mark.parametrize("w,steps", [
    (SOD_SMALL, 3),
    (workloads.variant(BURGERS, nx=40, x_lo=0.3, x_hi=0.9), 5),
    # N = 120, m = 3: 6 row tiles of 128 at n_pad = 128, two passes through tensor memory, H in HBM
    (workloads.variant(workloads.SOD_1D, nx=3, M=7, nq=8, x_lo=0.49, x_hi=0.51), 0),
], ids=["sod", "burgers", "sod_deg7_two_passes"])
def test_hessian_mixed_within_split_bound_fp64_exact(w, steps):
    prob = oracle_problem(w)
    st = _state_after(prob, steps)
    lam = st.lam[1:-1]
    ref = _packed(dual.dual_hessian(prob.space, prob.ent, lam))
    bound = 2.0 ** -12 * _abs_terms(prob, lam)
    for prec in ("fp64", "mixed"):
        ctx = gpu_context(w, precision=prec)
        ctx.set_moments(st.uhat)
        ctx.set_duals(st.lam)
        H = ctx.assemble_hessian()
        ctx.close()
        if prec == "fp64":
            assert rel_err(H, ref) < 1e-12
        else:
            err = np.abs(H - ref)
            assert np.all(err <= bound), float(np.max(err / np.maximum(bound, 1e-300)))
            # the split products are far more accurate than a single BF16 product (2^-8)
            assert rel_err(H, ref) < 1e-4


@pytest.mark.parametrize("w", [BURGERS, SOD_SMALL], ids=["burgers", "sod"])
def test_mixed_dual_solve_from_initial_data(w):
    prob = oracle_problem(w)
    st = s1.initial_state(prob)
    lam, it, stat, _ = dual.dual_solve(prob.space, prob.ent, st.lam[1:-1], st.uhat[1:-1], prob.newton)
    assert np.all(stat == 0)
    ctx = gpu_context(w, precision="mixed")
    s = ctx.dual_solve()
    assert s.failed_cells == 0 and s.tc_timeouts == 0
    g = ctx.get_duals()[1:-1]
    assert rel_err(g, lam) < TOL_MIXED
    # the FP64 stopping test still governs the result
    assert rel_err(g, lam) < 1e-9
    U = prob.ent.u_s(prob.space.evaluate(lam))
    assert rel_err(np.swapaxes(ctx.get_nodal_states()[1:-1], 1, 2), U) < TOL_MIXED
    # an approximate Hessian may cost extra Newton updates, never many
    assert s.newton_iters <= int(1.25 * it.sum()) + 2


def test_mixed_sod_steps_match_oracle():
    prob = oracle_problem(SOD_SMALL)
    st = s1.initial_state(prob)
    ctx = gpu_context(SOD_SMALL, precision="mixed")
    worst = 0.0
    for n in range(12):
        st = s1.ipm_step(prob, st)
        s = ctx.step()
        assert s.failed_cells == 0 and s.tc_timeouts == 0
        assert abs(s.dt - st.last_dt) <= 1e-6 * st.last_dt
        e = rel_err(ctx.get_moments(), st.uhat)
        worst = max(worst, e)
        assert e < TOL_MIXED, n
    assert worst < 1e-9


def test_mixed_burgers_full_run():
    prob = oracle_problem(BURGERS)
    ref = s1.run(prob)
    ctx = gpu_context(BURGERS, precision="mixed")
    s = ctx.run()
    assert s.failed_cells == 0 and s.tc_timeouts == 0
    assert s.steps == ref.n
    assert rel_err(ctx.get_moments(), ref.uhat) < TOL_MIXED


def test_mixed_oneshot_matches_oracle():
    w = workloads.variant(BURGERS, nx=30, M=4, nq=8, x_lo=0.0, x_hi=1.0, bc=("dirichlet", "outflow"),
                          u_minus=0.5, u_plus=4.0, t_end=0.0, x0=0.4, dx0=(0.1, 0, 0),
                          left=(2.0,), dleft=((0.5, 0, 0),), right=(3.0,), dright=((0.3, 0, 0),))
    prob = oracle_problem(w)
    st = s1.initial_state(prob)
    ctx = gpu_context(w, precision="mixed")
    for n in range(10):
        st = s1.oneshot_step(prob, st)
        s = ctx.oneshot_step()
        assert s.failed_cells == 0
    # One-Shot takes one damped step with the approximate Hessian: the iterates differ from the
    # FP64 ones by the Hessian error times the step, well inside the mixed tolerance
    assert rel_err(ctx.get_moments(), st.uhat) < TOL_MIXED
    assert rel_err(ctx.get_duals()[1:-1], st.lam[1:-1]) < 1e-4


def test_mixed_sod_full_size_first_step_sampled():
    """The 2000-cell Sod workload in mixed precision, first step, sampled cells (as for FP64)."""
    w = workloads.SOD_1D
    prob = oracle_problem(w)
    st = s1.initial_state(prob)
    ctx = gpu_context(w, precision="mixed")
    s = ctx.step()
    assert s.failed_cells == 0 and s.tc_timeouts == 0
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
