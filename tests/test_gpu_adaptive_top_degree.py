"""GPU parity of the top degree of the adaptive shear layer (Algorithm 3 with total degrees 2-6 in 3
uncertain dims, tensor Gauss 7^3 = 343 nodes) against the adaptive oracle, through the C ABI.

The cells at degree 6 carry N = 84 moments of m = 4 variables: N m = 336 unknowns, a packed Hessian
(455 KB) that lives in the per-CTA global workspace, and on the mixed path B N = 840 operand rows, i.e.
seven 128-row tensor-core tiles taken in two passes. The mesh is a thin periodic strip across the lower
edge of the dense band (y in [0.2, 0.3], band |y - 0.25| < 0.025 + 0.02 xi_3, same densities, velocities,
pressure and perturbation as the full shear layer), with cells fine enough against the edge's uncertain
range that most of them start at degree 6 (Eq. errorIndicator on the finest projection). The level change
rule, the level-wise Newton map and the mixed-degree update (Eq. adaptiveFVUpdate) are those of Sec. 5.

Levels are integers decided by FP64 comparisons on both sides and must agree exactly; moments to 1e-10
(FP64) or 1e-6 (mixed, and the FP32-factorisation mode); FP64 duals to 1e-9 and Newton counts exactly."""
import numpy as np
import pytest

from oracle import adaptive as ad
from paper_1912_09238_gb300 import workloads
from tests._cases import gpu_context, oracle_problem_2d, rel_err

pytestmark = pytest.mark.gpu

STRIP = workloads.variant(workloads.KH_2D, nx=4, ny=16, y_lo=0.2, y_hi=0.3, M=6, nq=7,
                          param=(0.01, 0.0, 0.025, 4.0 * np.pi))
LV = ad.Levels(degrees=(2, 3, 4, 5, 6), delta_lo=2e-5, delta_hi=2e-4)
TOP = 4                                  # level index of degree 6


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_09238_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def oracle_run():
    """Initial state and three Algorithm-3 steps of the oracle (computed once for the module)."""
    prob = oracle_problem_2d(STRIP)
    st = ad.initial_state(prob, LV)
    states = [st]
    for _ in range(3):
        st = ad.ipm_step(prob, st, LV)
        states.append(st)
    return states


def _grid(a, w):
    return a.reshape(w["ny"] + 2, w["nx"] + 2, *a.shape[1:])


@pytest.mark.parametrize("precision,steps,factorization", [("fp64", 3, 1), ("mixed", 3, 1), ("mixed_f32f", 1, 0),
                                                           ("fp64", 2, 2), ("mixed", 3, 2)],
                         ids=["fp64", "mixed", "mixed_f32f", "fp64_split", "mixed_split"])
def test_degree_six_cells_match_the_oracle(oracle_run, precision, steps, factorization):
    """factorization 1: blocked FP64 FMAs; 2: the split factorisation (tensor-core trailing updates)."""
    ctx = gpu_context(STRIP, precision=precision, adapt_min_degree=2, delta_lo=2e-5, delta_hi=2e-4,
                      factorization=factorization)
    d = ctx.dims
    assert (d.N, d.m, d.Q) == (84, 4, 343)
    st = oracle_run[0]
    assert np.array_equal(_grid(ctx.get_levels(), STRIP)[1:-1, 1:-1], st.level[1:-1, 1:-1])
    assert rel_err(_grid(ctx.get_moments(), STRIP)[1:-1, 1:-1], st.uhat[1:-1, 1:-1]) < 1e-13
    tol = 1e-10 if precision == "fp64" else 1e-6
    for n in range(steps):
        st = oracle_run[n + 1]
        s = ctx.step()
        assert s.failed_cells == 0 and s.tc_timeouts == 0, s.as_dict()
        lev = _grid(ctx.get_levels(), STRIP)[1:-1, 1:-1]
        assert np.array_equal(lev, st.level[1:-1, 1:-1]), n
        assert np.count_nonzero(lev == TOP) >= 16, n          # the path under test is taken every step
        assert rel_err(_grid(ctx.get_moments(), STRIP)[1:-1, 1:-1], st.uhat[1:-1, 1:-1]) < tol, n
        if precision == "fp64":
            assert rel_err(_grid(ctx.get_duals(), STRIP)[1:-1, 1:-1], st.lam[1:-1, 1:-1]) < 1e-9, n
            assert s.newton_iters == int(st.newton_iters.sum()), n
        if precision == "mixed_f32f":
            assert s.fp32_fallbacks == 0
    ctx.close()
