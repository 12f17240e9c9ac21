"""Frozen Hessians (ipm_options.hessian_reuse; the paper's outlook of quasi-Newton / frozen Hessians):
the kept Cholesky factor changes the iterates, not the fixed point, so the results meet the oracle's
Newton results at the precision path's tolerance with fewer factorisations."""
import numpy as np
import pytest

from oracle import scheme1d as s1
from paper_1912_09238_gb300 import workloads
from tests._cases import gpu_context, oracle_problem, rel_err

pytestmark = pytest.mark.gpu
SOD = workloads.variant(workloads.SOD_1D, nx=64)


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_09238_gb300 import build
    build.build()


@pytest.mark.parametrize("reuse", [1, 2])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_frozen_hessian_steps_reach_the_newton_results(reuse, precision):
    prob = oracle_problem(SOD)
    st = s1.initial_state(prob)
    ctx = gpu_context(SOD, precision=precision, hessian_reuse=reuse)
    iters = facts = 0
    for n in range(12):
        st = s1.ipm_step(prob, st)
        s = ctx.step()
        assert s.failed_cells == 0 and s.tc_timeouts == 0
        iters += s.newton_iters
        facts += s.factorizations
        # same stopping criterion, other iterates: agreement at the level the criterion fixes
        assert rel_err(ctx.get_moments(), st.uhat) < (1e-9 if precision == "fp64" else 1e-6), n
    assert facts < iters
    if reuse == 2:
        assert facts < 0.7 * iters


def test_newton_counts_one_factorisation_per_update():
    ctx = gpu_context(SOD)
    s = ctx.step()
    assert s.factorizations == s.newton_iters > 0


def test_kept_factors_are_refused_when_they_do_not_fit():
    from paper_1912_09238_gb300 import ipm
    with pytest.raises(ipm.IpmError) as e:
        gpu_context(workloads.variant(workloads.SOD_1D, nx=3_000_000), hessian_reuse=2)
    assert e.value.status == 1
