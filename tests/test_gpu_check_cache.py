"""Convergence checks from moment images (ipm_options.check_cache) through the C ABI: a context that
takes the first gradient of a solve from the cell's kept moment image gives bit-identical moments,
duals and Newton counts to one that evaluates every check, in every precision mode, after One-Shot
steps, with frozen Hessians, on 2-D meshes, and after the duals were changed from the host (the
images of the changed cells must not be used)."""
import numpy as np
import pytest

from paper_1912_09238_gb300 import workloads
from tests._cases import gpu_context

pytestmark = pytest.mark.gpu

SOD = workloads.variant(workloads.SOD_1D, nx=96, M=3, nq=4)          # N = 20, m = 3, Q = 64


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_09238_gb300 import build
    build.build()


def _pair(w, **kw):
    kw.setdefault("newton_kernel", 1)
    return gpu_context(w, check_cache=1, **kw), gpu_context(w, check_cache=0, **kw)


def _same(a, b):
    assert np.array_equal(a.get_moments(), b.get_moments())
    assert np.array_equal(a.get_duals(), b.get_duals())


def _steps(a, b, n, call="step"):
    cached = 0
    for _ in range(n):
        sa, sb = getattr(a, call)(), getattr(b, call)()
        assert sa.failed_cells == 0 and sb.failed_cells == 0
        assert (sa.newton_iters, sa.max_iters, sa.dt) == (sb.newton_iters, sb.max_iters, sb.dt)
        assert sb.cached_checks == 0
        cached += sa.cached_checks
    return cached


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_f32f"])
def test_identical_to_evaluating_every_check(precision):
    a, b = _pair(SOD, precision=precision)
    cached = _steps(a, b, 15)
    _same(a, b)
    assert np.array_equal(a.get_nodal_states(), b.get_nodal_states())
    assert cached > 5 * SOD["nx"]           # most cells of most steps are converged at their first check
    a.close()
    b.close()


def test_host_changed_duals_are_not_taken_from_the_image():
    a, b = _pair(SOD)
    _steps(a, b, 6)
    lam = a.get_duals()
    lam[10:20] *= 1.0 + 1e-7                # cells 10..19 no longer match their images
    a.set_duals(lam)
    b.set_duals(lam)
    sa, sb = a.step(), b.step()
    assert sa.newton_iters == sb.newton_iters and sa.cached_checks <= SOD["nx"] - 10
    _same(a, b)
    # the same duals written back unchanged keep every image usable
    a.set_duals(a.get_duals())
    b.set_duals(b.get_duals())
    _steps(a, b, 3)
    _same(a, b)
    a.close()
    b.close()


def test_after_oneshot_steps_and_with_frozen_hessians():
    a, b = _pair(SOD)
    _steps(a, b, 3, "oneshot_step")
    _steps(a, b, 4)
    _same(a, b)
    a.close()
    b.close()
    a, b = _pair(SOD, hessian_reuse=2)
    _steps(a, b, 8)
    _same(a, b)
    a.close()
    b.close()


def test_two_dimensional_mesh():
    w = workloads.variant(workloads.RAMP_2D, nx=16, ny=8, M=3, nq=4)
    a, b = _pair(w)
    _steps(a, b, 6)
    _same(a, b)
    a.close()
    b.close()


def test_checkpoint_restore_into_a_fresh_context():
    """A restored context has no images yet: its first solve evaluates every check and still continues
    bit for bit."""
    a, b = _pair(SOD)
    _steps(a, b, 5)
    mom, lam = a.get_moments(), a.get_duals()
    c = gpu_context(SOD, newton_kernel=1, check_cache=1)
    c.set_moments(mom)
    c.set_duals(lam)
    sa, sc = a.step(), c.step()
    assert sc.cached_checks == 0 and sa.newton_iters == sc.newton_iters
    _same(a, c)
    for x in (a, b, c):
        x.close()


def test_headline_workload_full_size():
    """The 2000-cell Sod workload in mixed precision, in the launch configuration the bench times: ten
    steps with images against ten without, bit for bit (the first step is checked against the oracle
    on sampled cells in test_gpu_mixed_1d)."""
    a = gpu_context(workloads.SOD_1D, precision="mixed", check_cache=1)
    b = gpu_context(workloads.SOD_1D, precision="mixed", check_cache=0)
    cached = _steps(a, b, 10)
    _same(a, b)
    assert cached > 8 * 1500
    a.close()
    b.close()


ADAPTIVE = [
    # shear layer: the transverse perturbation moves every cell, so few checks come from images
    (workloads.variant(workloads.KH_2D, nx=16, ny=16, M=4, nq=5), dict(delta_lo=2e-4, delta_hi=2e-5), 0),
    # ramp: the freestream ahead of the shock is settled after a few steps
    (workloads.variant(workloads.RAMP_2D, nx=16, ny=8, M=4, nq=5), dict(delta_lo=1e-10, delta_hi=1e-8), 1),
]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ADAPTIVE, ids=["shear_layer", "ramp"])
def test_adaptive_degrees_on_one_rule(precision, case):
    """Adaptive degrees (Algorithm 3) with the shared Gauss rule: the images carry the level they were
    taken at, so a cell whose level changed is evaluated; the degree-2 cells (one warp per cell, nodes in
    chunks) and the others (one CTA per cell) both use them. Levels, moments and duals bit for bit."""
    w, lv, min_cached = case
    kw = dict(precision=precision, adapt_min_degree=2, **lv)
    a, b = gpu_context(w, check_cache=1, **kw), gpu_context(w, check_cache=0, **kw)
    cached = 0
    for _ in range(8):
        sa, sb = a.step(), b.step()
        assert sa.failed_cells == 0 and (sa.newton_iters, sa.dt) == (sb.newton_iters, sb.dt)
        assert np.array_equal(a.get_levels(), b.get_levels())
        cached += sa.cached_checks
    _same(a, b)
    assert cached >= min_cached
    a.close()
    b.close()


def test_per_level_rules_do_not_use_images():
    w = workloads.variant(workloads.KH_2D, nx=10, ny=10, M=3, nq=3, p=2, cc_levels=(1, 2, 2),
                          dparam=((0.005, 0.0, 0.0), (0.0, 0.1, 0.0), (0.05, 0.0, 0.0), (0.0, 0.0, 0.0)))
    ctx = gpu_context(w, adapt_min_degree=1, delta_lo=2e-5, delta_hi=2e-4)
    for _ in range(3):
        assert ctx.step().cached_checks == 0
    ctx.close()
