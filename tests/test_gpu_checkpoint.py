"""Checkpoint / resume through the C ABI (ipm_get_state / ipm_set_state): a fresh context restored from
a checkpoint continues bit for bit as the original context does (FP64 and mixed, 1-D and an
adaptive 2-D mesh), because no result of a step depends on which CTA or warp takes which cell."""
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


CASES = [
    (workloads.variant(workloads.SOD_1D, nx=64, t_end=0.14), "fp64", {}),
    (workloads.variant(workloads.SOD_1D, nx=64, t_end=0.14), "mixed", {}),
    (workloads.variant(workloads.KH_2D, nx=12, ny=12, M=4, nq=5), "fp64",
     dict(adapt_min_degree=2, delta_lo=2e-4, delta_hi=2e-5)),
]


@pytest.mark.parametrize("w,prec,opt", CASES, ids=["sod_fp64", "sod_mixed", "shear_adaptive"])
def test_resume_continues_bit_for_bit(w, prec, opt):
    a = gpu_context(w, precision=prec, **opt)
    for _ in range(3):
        assert a.step().failed_cells == 0
    m, d, lv, ck = a.get_state(levels=True, clock=True)
    assert ck.steps == 3 and ck.t > 0.0
    for _ in range(4):
        sa = a.step()
    b = gpu_context(w, precision=prec, **opt)
    b.set_state(m, d, levels=lv, clock=ck)
    for _ in range(4):
        sb = b.step()
    assert np.array_equal(a.get_moments(), b.get_moments())
    assert np.array_equal(a.get_duals(), b.get_duals())
    if opt:
        assert np.array_equal(a.get_levels(), b.get_levels())
    assert sa.t == sb.t and sa.steps == sb.steps and sa.dt == sb.dt
    a.close()
    b.close()


def test_state_checks():
    w = workloads.variant(workloads.KH_2D, nx=6, ny=6, M=3, nq=4)
    ctx = gpu_context(w, adapt_min_degree=2)
    m, d, lv = ctx.get_state(levels=True)
    with pytest.raises(ipm.IpmError):
        ctx.set_state(m, d, levels=np.full_like(lv, 7))          # above the finest level
    with pytest.raises(ValueError):
        ctx.get_state(np.empty(3), d)
    ctx.set_state(m, d, levels=lv)
    ctx.close()
