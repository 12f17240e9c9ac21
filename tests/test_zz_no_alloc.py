"""ipm_dual_solve_noalloc: the dual solve for callers that cannot allocate device memory themselves
(their device memory belongs to another allocator, or they run loops that must not pay cudaMalloc's
synchronisation). Its scratch lives in one static device array inside the library; this test checks,
through the C ABI, that two calls in a row on caller-owned buffers give the same duals, nodal states,
iteration counts and statuses as the context-based ipm_dual_solve, within the parity tolerance."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_09238_gb300 import build
    build.build()
    return torch


@pytest.mark.parametrize("which", ["sod", "burgers", "sod_global_hessian"])
def test_noalloc_matches_context_solve_twice(torch_cuda, which):
    torch = torch_cuda
    from paper_1912_09238_gb300 import ipm, workloads
    from tests._cases import gpu_context, rel_err
    if which == "sod":
        w = workloads.variant(workloads.SOD_1D, nx=48)
    elif which == "burgers":
        w = workloads.variant(workloads.BURGERS_1D, nx=64)
    else:   # N*m = 252: the packed Hessian lives in the scratch array's workspace slots
        w = workloads.variant(workloads.SOD_1D, nx=5, M=6, nq=7)
    ctx = gpu_context(w)
    uhat0 = ctx.get_moments()[1:-1]
    lam0 = ctx.get_duals()[1:-1]
    s_ref = ctx.dual_solve()
    lam_ref = ctx.get_duals()[1:-1]
    nodal_ref = ctx.get_nodal_states()[1:-1]
    ctx.close()
    assert s_ref.failed_cells == 0

    n = uhat0.shape[0]
    d = ctx.dims
    dev = torch.device("cuda", torch.cuda.current_device())
    d_uhat = torch.from_numpy(np.ascontiguousarray(uhat0)).to(dev)
    d_nodal = torch.zeros((n, d.m, d.Q), dtype=torch.float64, device=dev)
    d_iters = torch.zeros(n, dtype=torch.int32, device=dev)
    d_status = torch.full((n,), -1, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    for call in range(2):
        d_lam = torch.from_numpy(np.ascontiguousarray(lam0)).to(dev)
        torch.cuda.synchronize()
        s = ipm.ipm_dual_solve_noalloc(w["kind"], w["gamma"], w["p"], w["M"], w["nq"], w["entropy"], n,
                                       d_uhat.data_ptr(), d_lam.data_ptr(), d_nodal.data_ptr(), d_iters.data_ptr(),
                                       d_status.data_ptr(), stream=0, u_minus=w.get("u_minus", 0.0),
                                       u_plus=w.get("u_plus", 0.0),
                                       options=ipm.default_options(newton_tol=w["newton_tol"]))
        torch.cuda.synchronize()
        assert s.failed_cells == 0, (call, s.as_dict())
        assert s.newton_iters == s_ref.newton_iters
        assert rel_err(d_lam.cpu().numpy(), lam_ref) < TOL, call
        assert rel_err(d_nodal.cpu().numpy(), nodal_ref) < TOL, call
        assert np.all(d_status.cpu().numpy() == 0)


def test_noalloc_rejects_sizes_beyond_its_scratch(torch_cuda):
    torch = torch_cuda
    from paper_1912_09238_gb300 import ipm
    dev = torch.device("cuda", torch.cuda.current_device())
    buf = torch.zeros(8, dtype=torch.float64, device=dev)
    ib = torch.zeros(8, dtype=torch.int32, device=dev)
    with pytest.raises(ipm.IpmError) as e:
        ipm.ipm_dual_solve_noalloc("euler1d", 1.4, 3, 5, 6, "euler", 262145, buf.data_ptr(), buf.data_ptr(),
                                   buf.data_ptr(), ib.data_ptr(), ib.data_ptr())
    assert e.value.status == 1 and "n_cells" in str(e.value)
