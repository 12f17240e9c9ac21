"""GPU parity of adaptive IPM (Algorithm 3, per-cell total degree from Eq. errorIndicator) against the
adaptive oracle, on the periodic shear-layer workload at reduced size, through the C ABI.

The levels are integers decided by FP64 comparisons on both sides and must agree exactly; moments
and duals to 1e-10 (FP64 path) or 1e-6 (mixed path)."""
import numpy as np
import pytest

from oracle import adaptive as ad
from paper_1912_09238_gb300 import workloads
from tests._cases import gpu_context, oracle_problem_2d, rel_err

pytestmark = pytest.mark.gpu

KH = workloads.variant(workloads.KH_2D, nx=12, ny=12, M=4, nq=5)
LV = ad.Levels(degrees=(2, 3, 4), delta_lo=2e-4, delta_hi=2e-5)


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_09238_gb300 import build
    build.build()


def _grid(a, w):
    return a.reshape(w["ny"] + 2, w["nx"] + 2, *a.shape[1:])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_adaptive_steps_match_the_oracle(precision):
    prob = oracle_problem_2d(KH)
    st = ad.initial_state(prob, LV)
    ctx = gpu_context(KH, precision=precision, adapt_min_degree=2, delta_lo=2e-4, delta_hi=2e-5)
    tol = 1e-10 if precision == "fp64" else 1e-6
    assert np.array_equal(_grid(ctx.get_levels(), KH)[1:-1, 1:-1], st.level[1:-1, 1:-1])
    assert rel_err(_grid(ctx.get_moments(), KH)[1:-1, 1:-1], st.uhat[1:-1, 1:-1]) < 1e-13
    seen = set()
    for n in range(5):
        st = ad.ipm_step(prob, st, LV)
        s = ctx.step()
        assert s.failed_cells == 0 and s.tc_timeouts == 0
        lev = _grid(ctx.get_levels(), KH)[1:-1, 1:-1]
        assert np.array_equal(lev, st.level[1:-1, 1:-1]), n
        seen |= set(np.unique(lev).tolist())
        assert rel_err(_grid(ctx.get_moments(), KH)[1:-1, 1:-1], st.uhat[1:-1, 1:-1]) < tol, n
        if precision == "fp64":
            assert rel_err(_grid(ctx.get_duals(), KH)[1:-1, 1:-1], st.lam[1:-1, 1:-1]) < 1e-9
            assert s.newton_iters == int(st.newton_iters.sum())
    assert len(seen) >= 2                      # the levels did change


def test_adaptive_rejects_1d_and_bad_ranges():
    from paper_1912_09238_gb300 import ipm
    with pytest.raises(ipm.IpmError):
        gpu_context(workloads.variant(workloads.BURGERS_1D, nx=10), adapt_min_degree=2)
    with pytest.raises(ipm.IpmError):
        gpu_context(KH, adapt_min_degree=5)       # above the basis degree


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_retarded_adaptive_oneshot_matches_the_oracle(precision):
    """Algorithm 4 on a coarse ramp mesh: stages, levels, steps and moments as the oracle."""
    w = workloads.variant(workloads.RAMP_2D, nx=10, ny=5, M=4, nq=5)
    prob = oracle_problem_2d(w)
    lv = ad.Levels(degrees=(2, 3, 4), delta_lo=1e-10, delta_hi=1e-8)
    st, hist = ad.oneshot_retarded(prob, lv, caps=(0, 2), tolerances=(2e-3,), tol=1e-9, max_steps=40)
    ctx = gpu_context(w, precision=precision, adapt_min_degree=2, delta_lo=1e-10, delta_hi=1e-8)
    s = ctx.oneshot_retarded([0, 2], [2e-3], 1e-9, 40)
    assert s.failed_cells == 0
    assert s.steps == st.n
    assert np.array_equal(_grid(ctx.get_levels(), w)[1:-1, 1:-1], st.level[1:-1, 1:-1])
    tol = 1e-10 if precision == "fp64" else 1e-6
    assert rel_err(_grid(ctx.get_moments(), w)[1:-1, 1:-1], st.uhat[1:-1, 1:-1]) < tol


# ---------- a quadrature rule per refinement level (nested Clenshaw-Curtis) ----------
KH_CC = workloads.variant(workloads.KH_2D, nx=10, ny=10, M=3, nq=3, p=2, cc_levels=(1, 2, 2),
                          dparam=((0.005, 0.0, 0.0), (0.0, 0.1, 0.0), (0.05, 0.0, 0.0), (0.0, 0.0, 0.0)))
LV_CC = ad.Levels(degrees=(1, 2, 3), delta_lo=2e-5, delta_hi=2e-4, quad_levels=(1, 2, 2))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_per_level_rules_match_the_oracle(precision):
    """Degrees 1-3 on the 3-, 5- and 5-point Clenshaw-Curtis rules (9, 25, 25 nodes): every cell's dual
    problem on its level's rule, updates on the new level's rule with coarser neighbours evaluated at
    the finer nodes; levels exact, moments to the precision's tolerance, dt to rounding."""
    prob = oracle_problem_2d(KH_CC)
    st = ad.initial_state(prob, LV_CC)
    ctx = gpu_context(KH_CC, precision=precision, adapt_min_degree=1, delta_lo=2e-5, delta_hi=2e-4)
    tol = 1e-10 if precision == "fp64" else 1e-6
    assert ctx.dims.Q == 25
    assert np.array_equal(_grid(ctx.get_levels(), KH_CC)[1:-1, 1:-1], st.level[1:-1, 1:-1])
    assert rel_err(_grid(ctx.get_moments(), KH_CC)[1:-1, 1:-1], st.uhat[1:-1, 1:-1]) < 1e-13
    seen = set()
    for n in range(4):
        st = ad.ipm_step(prob, st, LV_CC)
        s = ctx.step()
        assert s.failed_cells == 0 and s.tc_timeouts == 0
        assert abs(s.dt - st.last_dt) <= 1e-12 * st.last_dt
        lev = _grid(ctx.get_levels(), KH_CC)[1:-1, 1:-1]
        assert np.array_equal(lev, st.level[1:-1, 1:-1]), n
        seen |= set(np.unique(lev).tolist())
        assert rel_err(_grid(ctx.get_moments(), KH_CC)[1:-1, 1:-1], st.uhat[1:-1, 1:-1]) < tol, n
        if precision == "fp64":
            assert rel_err(_grid(ctx.get_duals(), KH_CC)[1:-1, 1:-1], st.lam[1:-1, 1:-1]) < 1e-9
    assert len(seen) >= 2


def test_per_level_rules_on_the_ramp_with_dirichlet_ghosts():
    """The 2-D ramp with Dirichlet ghosts at their own level's rule, One-Shot steps with per-level rules
    (degrees 2-4 on Clenshaw-Curtis levels 2, 2, 3: 25, 25, 81 nodes)."""
    w = workloads.variant(workloads.RAMP_2D, nx=10, ny=5, M=4, nq=5, cc_levels=(2, 2, 3))
    prob = oracle_problem_2d(w)
    lv = ad.Levels(degrees=(2, 3, 4), delta_lo=1e-10, delta_hi=1e-8, quad_levels=(2, 2, 3))
    st = ad.initial_state(prob, lv)
    ctx = gpu_context(w, adapt_min_degree=2, delta_lo=1e-10, delta_hi=1e-8)
    for n in range(6):
        st = ad.oneshot_step(prob, st, lv, 2)
        s = ctx.oneshot_step()
        assert s.failed_cells == 0
        assert np.array_equal(_grid(ctx.get_levels(), w)[1:-1, 1:-1], st.level[1:-1, 1:-1]), n
        assert rel_err(_grid(ctx.get_moments(), w)[1:-1, 1:-1], st.uhat[1:-1, 1:-1]) < 1e-10, n


def test_clenshaw_curtis_rule_checks():
    from paper_1912_09238_gb300 import ipm
    with pytest.raises(ipm.IpmError):           # decreasing levels
        gpu_context(workloads.variant(KH_CC, cc_levels=(2, 1, 2)), adapt_min_degree=1)
    with pytest.raises(ipm.IpmError):           # 3 points per dimension cannot carry degree 3
        gpu_context(workloads.variant(KH_CC, cc_levels=(1, 1, 1)), adapt_min_degree=1)
    # all zero: the default rule (smallest level with 2^k + 1 >= degree + 2): 1, 2, 2 for degrees 1-3
    ctx = gpu_context(workloads.variant(KH_CC, cc_levels=()), adapt_min_degree=1, delta_lo=2e-5, delta_hi=2e-4)
    ref = gpu_context(KH_CC, adapt_min_degree=1, delta_lo=2e-5, delta_hi=2e-4)
    ctx.step()
    ref.step()
    assert np.array_equal(ctx.get_moments(), ref.get_moments())


@pytest.mark.parametrize("w", [KH, KH_CC], ids=["gauss", "clenshaw_curtis"])
def test_small_cells_on_the_warp_kernel_equal_the_cta_kernel(w):
    """The lowest levels (N m <= 64) run one warp per cell beside the CTA-per-cell kernel; forcing every
    cell onto the CTA kernel (newton_kernel = 1) gives the same levels and moments to rounding."""
    kw = dict(adapt_min_degree=2, delta_lo=2e-4, delta_hi=2e-5) if w is KH else dict(adapt_min_degree=1, delta_lo=2e-5,
                                                                                      delta_hi=2e-4)
    split = gpu_context(w, **kw)
    cta = gpu_context(w, newton_kernel=1, **kw)
    for _ in range(3):
        a, b = split.step(), cta.step()
        assert a.failed_cells == 0 and b.failed_cells == 0
        assert a.newton_iters == b.newton_iters
        assert np.array_equal(split.get_levels(), cta.get_levels())
        assert rel_err(split.get_moments(), cta.get_moments()) < 1e-12
