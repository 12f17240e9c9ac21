"""The 1-D Lax-Friedrichs update folded into the Newton launch (A_j - dt/dx B_j, formed by the CTA that
finishes the last neighbour of cell j) against the stand-alone update kernel with the same dt, through
the C ABI: the same moments to rounding after several steps, on both Newton kernels (one CTA or one
warp per cell), for every boundary condition and for meshes of one to three cells (whose neighbours
are the cell itself, the other end or fixed ghosts)."""
import pytest

from paper_1912_09238_gb300 import workloads
from tests._cases import gpu_context, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_09238_gb300 import build
    build.build()


def _compare(w, steps, precision="fp64", tol=1e-10, **opt):
    folded = gpu_context(w, precision=precision, **opt)
    plain = gpu_context(w, precision=precision, **opt)
    for _ in range(steps):
        s = folded.step()
        assert s.failed_cells == 0 and s.dt > 0.0
        assert plain.dual_solve().failed_cells == 0
        plain.update(s.dt)
        err = rel_err(folded.get_moments(), plain.get_moments())
        assert err < tol, err
    folded.close()
    plain.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sod_outflow(precision):
    _compare(workloads.variant(workloads.SOD_1D, nx=120), 6, precision)


@pytest.mark.parametrize("kernel", [1, 2], ids=["cta_per_cell", "warp_per_cell"])
@pytest.mark.parametrize("bc", [("periodic", "periodic"), ("dirichlet", "outflow"), ("outflow", "dirichlet")])
def test_burgers_boundaries(bc, kernel):
    _compare(workloads.variant(workloads.BURGERS_1D, nx=60, bc=bc, x0=0.4), 8, newton_kernel=kernel)


@pytest.mark.parametrize("kernel", [1, 2], ids=["cta_per_cell", "warp_per_cell"])
@pytest.mark.parametrize("nx", [1, 2, 3])
@pytest.mark.parametrize("bc", [("periodic", "periodic"), ("dirichlet", "dirichlet"), ("outflow", "outflow")])
def test_tiny_meshes(nx, bc, kernel):
    # one cell spans the whole interval: a long end time keeps dt > 0 for every step compared
    _compare(workloads.variant(workloads.BURGERS_1D, nx=nx, bc=bc, t_end=100.0), 3, newton_kernel=kernel)


def test_mixed_warp_kernel():
    _compare(workloads.variant(workloads.BURGERS_1D, nx=200), 10, "mixed", newton_kernel=2)
