"""The split Cholesky factorisation (ipm_options.factorization = 2): panels of 16 columns in FP64 and
every trailing update L21 L21^T as exact integer products of base-256 digit slices on the tensor cores.

Checked through the C ABI: (1) its factors of the Hessians the Newton kernel assembles have the
backward error of an FP64 factorisation (|L L^T - H| / |H| at rounding level, like the blocked FP64-FMA
factorisation's), in both precision modes, for N m = 168 (shared-memory Hessian) and 336 (workspace
Hessian); (2) Algorithm-1 runs with it match the oracle to the precision's tolerance (1e-10 FP64 Hessian,
1e-6 split-BF16 Hessian) with the FP64 path's Newton counts; (3) frozen Hessians keep working on its
factors."""
import numpy as np
import pytest

from oracle import scheme1d as s1
from paper_1912_09238_gb300 import workloads
from tests._cases import gpu_context, oracle_problem, rel_err

pytestmark = pytest.mark.gpu

SOD = workloads.variant(workloads.SOD_1D, nx=40, x_lo=0.4, x_hi=0.6)      # N m = 168, cells across the jump
SOD_BIG = workloads.variant(workloads.SOD_1D, nx=6, x_lo=0.45, x_hi=0.55, M=6, nq=7, p=3)   # N m = 252


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_09238_gb300 import build
    build.build()


def _unpack(packed, n):
    L = np.zeros((n, n))
    L[np.tril_indices(n)] = packed
    return L


def _backward_errors(ctx):
    d = ctx.dims
    n = d.N * d.m
    H = ctx.assemble_hessian()
    F = ctx.factor_hessian()
    s = ctx.sync_stats()
    assert s.failed_cells == 0, s.as_dict()
    out = []
    for h, f in zip(H, F):
        Hm = _unpack(h, n)
        Hm = Hm + np.tril(Hm, -1).T
        L = _unpack(f, n)
        out.append(np.abs(L @ L.T - Hm).max() / np.abs(Hm).max())
    return np.array(out), H


@pytest.mark.parametrize("w", [SOD, SOD_BIG], ids=["nm168", "nm252"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_split_factor_has_fp64_backward_error(w, precision):
    ctx = gpu_context(w, precision=precision, factorization=2)
    ref = gpu_context(w, precision=precision, factorization=1)
    ref.dual_solve()                       # a converged state: Hessians of every kind of cell in the window
    ctx.set_duals(ref.get_duals())         # both factorisations at the same duals
    be, H = _backward_errors(ctx)
    be_ref, H_ref = _backward_errors(ref)
    assert np.array_equal(H, H_ref)        # the same Hessians go into both factorisations
    # FP64 rounding level of an n = 168..252 factorisation (the FMA factorisation's own is ~1e-16)
    assert be.max() < 2e-14, be.max()
    assert be.max() < 50 * max(be_ref.max(), 1e-16), (be.max(), be_ref.max())


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-6)])
def test_split_factor_steps_match_the_oracle(precision, tol):
    prob = oracle_problem(SOD)
    st = s1.initial_state(prob)
    ctx = gpu_context(SOD, precision=precision, factorization=2)
    plain = gpu_context(SOD, precision="fp64", factorization=1)
    for n in range(4):
        st = s1.ipm_step(prob, st)
        s = ctx.step()
        sp = plain.step()
        assert s.failed_cells == 0 and s.tc_timeouts == 0, s.as_dict()
        assert rel_err(ctx.get_moments(), st.uhat) < tol, n
        if precision == "fp64":
            assert rel_err(ctx.get_duals(), st.lam) < 1e-9, n
            # the two GPU factorisations take the same updates; a cell whose residual lands at the stopping
            # threshold may take one update more or less than in the oracle's rounding order
            assert s.newton_iters == sp.newton_iters, n
            assert abs(s.newton_iters - int(st.newton_iters.sum())) <= 2, n


def test_split_factor_is_the_mixed_default_for_large_systems():
    """factorization = 0 takes the split factorisation on IPM_PREC_MIXED for N m >= 128: bit-identical
    to asking for it, and different in rounding from the FMA factorisation."""
    a = gpu_context(SOD, precision="mixed")
    b = gpu_context(SOD, precision="mixed", factorization=2)
    c = gpu_context(SOD, precision="mixed", factorization=1)
    for _ in range(3):
        a.step(), b.step(), c.step()
    assert np.array_equal(a.get_moments(), b.get_moments())
    assert rel_err(a.get_moments(), c.get_moments()) < 1e-9


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_split_factor_with_frozen_hessians(precision):
    """hessian_reuse = 2 keeps the split factors between solves; the fixed point is the Newton one."""
    prob = oracle_problem(SOD)
    st = s1.initial_state(prob)
    ctx = gpu_context(SOD, precision=precision, factorization=2, hessian_reuse=2)
    for n in range(4):
        st = s1.ipm_step(prob, st)
        s = ctx.step()
        assert s.failed_cells == 0
        assert rel_err(ctx.get_moments(), st.uhat) < (1e-9 if precision == "fp64" else 1e-6), n


def test_split_factor_option_checks():
    from paper_1912_09238_gb300 import ipm
    with pytest.raises(ipm.IpmError):
        gpu_context(SOD, precision="mixed_f32f", factorization=2)
    with pytest.raises(ipm.IpmError):
        gpu_context(SOD, precision="mixed", factorization=3)
