"""The warp-per-cell Newton kernel (cells with N*m <= 64) against the oracle, forced through the
ipm_options.newton_kernel switch, next to the CTA-per-cell kernel; and the autotuner's report."""
import numpy as np
import pytest

from oracle import dual
from oracle import scheme1d as s1
from oracle import scheme2d as s2
from paper_1912_09238_gb300 import workloads
from tests._cases import gpu_context, oracle_problem, oracle_problem_2d, rel_err

pytestmark = pytest.mark.gpu
KERNELS = {"cta": 1, "warp": 2}


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_09238_gb300 import build
    build.build()


@pytest.mark.parametrize("kernel", ["cta", "warp"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_burgers_full_run(kernel, precision):
    w = workloads.BURGERS_1D
    prob = oracle_problem(w)
    ref = s1.run(prob)
    ctx = gpu_context(w, precision=precision, newton_kernel=KERNELS[kernel])
    assert ctx.tuning()[0] == KERNELS[kernel]
    s = ctx.run()
    assert s.failed_cells == 0 and s.steps == ref.n
    assert rel_err(ctx.get_moments(), ref.uhat) < (1e-10 if precision == "fp64" else 1e-6)


@pytest.mark.parametrize("kernel", ["cta", "warp"])
def test_sod_low_degree_steps_and_dirichlet(kernel):
    w = workloads.variant(workloads.SOD_1D, nx=50, M=2, nq=3, bc=("dirichlet", "outflow"))     # N*m = 30
    prob = oracle_problem(w)
    st = s1.initial_state(prob)
    ctx = gpu_context(w, newton_kernel=KERNELS[kernel])
    for n in range(8):
        st = s1.ipm_step(prob, st)
        s = ctx.step()
        assert s.failed_cells == 0
        assert s.newton_iters == int(st.newton_iters[1:-1].sum())
        assert rel_err(ctx.get_moments(), st.uhat) < 1e-10, n


@pytest.mark.parametrize("kernel", ["cta", "warp"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_2d_ramp_oneshot_and_shear_steps(kernel, precision):
    tol = 1e-10 if precision == "fp64" else 1e-6
    w = workloads.variant(workloads.RAMP_2D, nx=16, ny=8, M=2, nq=3)                        # N*m = 24
    prob = oracle_problem_2d(w)
    st = s2.initial_state(prob)
    ctx = gpu_context(w, precision=precision, newton_kernel=KERNELS[kernel])
    for _ in range(10):
        st = s2.oneshot_step(prob, st)
        assert ctx.oneshot_step().failed_cells == 0
    got = ctx.get_moments().reshape(st.uhat.shape)
    assert rel_err(got[1:-1, 1:-1], st.uhat[1:-1, 1:-1]) < tol
    w = workloads.variant(workloads.KH_2D, nx=10, ny=10, M=2, nq=3)                          # N*m = 40
    prob = oracle_problem_2d(w)
    st = s2.initial_state(prob)
    ctx = gpu_context(w, precision=precision, newton_kernel=KERNELS[kernel])
    for _ in range(3):
        st = s2.ipm_step(prob, st)
        assert ctx.step().failed_cells == 0
    got = ctx.get_moments().reshape(st.uhat.shape)
    assert rel_err(got[1:-1, 1:-1], st.uhat[1:-1, 1:-1]) < tol


def test_warp_kernel_reports_infeasible_cells():
    w = workloads.variant(workloads.SOD_1D, nx=8, M=2, nq=3)
    ctx = gpu_context(w, newton_kernel=2)
    lam = ctx.get_duals()
    lam[3, 0, 2] = abs(lam[3, 0, 2]) * 10 + 5.0          # Lambda_E > 0 at every node of cell 3
    ctx.set_duals(lam)
    s = ctx.dual_solve()
    assert s.failed_cells == 1 and s.first_failed_cell == 3 and s.first_status == 5


def test_autotuner_times_both_variants_and_refuses_a_forced_misfit():
    from paper_1912_09238_gb300 import ipm
    ctx = gpu_context(workloads.variant(workloads.RAMP_2D, nx=64, ny=32, M=4, nq=5))      # N*m = 60
    kind, ms_cta, ms_warp = ctx.tuning()
    assert kind in (1, 2) and ms_cta > 0 and ms_warp > 0
    assert (kind == 2) == (ms_warp < 0.97 * ms_cta)
    with pytest.raises(ipm.IpmError):
        gpu_context(workloads.variant(workloads.SOD_1D, nx=20), newton_kernel=2)           # N*m = 168
