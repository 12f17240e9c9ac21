"""Failure handling through the C ABI, made on the host (nothing here faults, traps or hangs a GPU):
device allocations that cannot succeed return IPM_ENOMEM and leave the device usable; non-finite or
non-realisable moments written from the host become per-cell status words while the other cells
are solved and the context stays usable."""
import numpy as np
import pytest

from paper_1912_09238_gb300 import ipm, workloads
from tests._cases import gpu_context

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_09238_gb300 import build
    build.build()


def test_device_allocation_failure_is_enomem_and_the_device_stays_usable():
    # 3e8 Sod cells need ~400 GB for the moments alone: the first large allocation fails cleanly
    with pytest.raises(ipm.IpmError) as e:
        gpu_context(workloads.variant(workloads.SOD_1D, nx=300_000_000))
    assert e.value.status == 2                                   # IPM_ENOMEM
    ctx = gpu_context(workloads.variant(workloads.SOD_1D, nx=16, M=2, nq=3))
    assert ctx.step().failed_cells == 0
    ctx.close()


def test_non_finite_moments_are_a_cell_status_not_a_failure():
    w = workloads.variant(workloads.SOD_1D, nx=12, M=2, nq=3)
    ctx = gpu_context(w)
    good = ctx.get_moments()
    bad = good.copy()
    bad[5, 1, 0] = np.nan
    ctx.set_moments(bad)
    s = ctx.dual_solve()
    assert s.failed_cells == 1 and s.first_failed_cell == 5 and s.first_status == 7   # IPM_ENONFINITE
    # the context is still usable: restore the moments and solve again
    ctx.set_moments(good)
    assert ctx.dual_solve().failed_cells == 0
    ctx.close()


def test_non_realisable_moments_are_reported():
    """A negative mean density has no entropy-admissible state: the dual problem of that cell fails
    (unbounded below, or a line search or feasibility failure) and is reported per cell."""
    w = workloads.variant(workloads.SOD_1D, nx=12, M=2, nq=3)
    ctx = gpu_context(w)
    m = ctx.get_moments()
    m[4, 0, 0] = -abs(m[4, 0, 0])
    ctx.set_moments(m)
    s = ctx.dual_solve()
    assert s.failed_cells >= 1 and s.first_failed_cell == 4 and s.first_status in (3, 4, 5, 6, 7)
    ctx.close()
