"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads, exports every entry point
declared in include/ipm.h, and its host-built tables agree with the oracle's independent ones."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libipm():
    from paper_1912_09238_gb300 import build, ipm
    build.build()
    return ipm.lib()


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(ipm_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(libipm):
    from paper_1912_09238_gb300 import ipm
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(libipm, n), n
    bound = {s[0] for s in ipm.SIGNATURES}
    assert set(names) <= bound, set(names) - bound


@pytest.mark.parametrize("p,M,nq", [(1, 5, 10), (3, 5, 6), (2, 4, 5), (3, 2, 3), (1, 0, 1)])
def test_library_tables_match_oracle(libipm, p, M, nq):
    from oracle.basis import StochasticSpace
    from paper_1912_09238_gb300 import ipm
    idx, nodes, w, phi = ipm.ipm_tables(p, M, nq)
    sp = StochasticSpace(p, M, nq)
    assert np.array_equal(idx, sp.indices)
    np.testing.assert_allclose(nodes, sp.nodes, rtol=0, atol=4e-16)
    np.testing.assert_allclose(w, sp.w, rtol=1e-14, atol=0)
    np.testing.assert_allclose(phi, sp.Phi, rtol=0, atol=5e-14)


def test_tables_reject_bad_sizes(libipm):
    import ctypes
    n = ctypes.c_int()
    q = ctypes.c_int()
    assert libipm.ipm_tables(0, 3, 3, 10, 10, None, None, None, None, ctypes.byref(n), ctypes.byref(q)) == 1
    assert libipm.ipm_tables(4, 3, 3, 10, 10, None, None, None, None, ctypes.byref(n), ctypes.byref(q)) == 1


def test_init_without_a_gpu_fails_cleanly(libipm):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1912_09238_gb300 import ipm, workloads
    from tests._cases import gpu_context
    with pytest.raises(ipm.IpmError) as e:
        gpu_context(workloads.BURGERS_1D)
    assert e.value.status in (9, 1)


@pytest.mark.parametrize("p,M,kmax", [(1, 4, 3), (2, 3, 2), (3, 2, 2)])
def test_library_clenshaw_curtis_tables_match_oracle(libipm, p, M, kmax):
    """The library's nested Clenshaw-Curtis tables (weights from a Chebyshev moment solve) against the
    oracle's (closed-form weights): same node order, nodes, every level's weights, basis values."""
    from oracle import basis as ob
    from paper_1912_09238_gb300 import ipm
    idx, nodes, lw, phi = ipm.ipm_tables_cc(p, M, kmax)
    onodes, _, ow = ob.nested_cc_tensor(p, kmax)
    assert np.abs(nodes - onodes).max() < 1e-15
    for k in range(kmax + 1):
        assert np.abs(lw[k, :ow[k].size] - ow[k]).max() < 1e-15
        assert np.all(lw[k, ow[k].size:] == 0.0)
    sp = ob.NestedCCSpace(p, M, kmax)
    assert np.array_equal(idx, sp.indices) and np.abs(phi - sp.Phi).max() < 1e-13


def test_option_defaults_and_validation_without_a_gpu(libipm):
    """ipm_default_options through the ctypes mirror of ipm_options (a layout mismatch would show as
    wrong defaults), and option checks that refuse a plan before any device work."""
    import ctypes
    from paper_1912_09238_gb300 import ipm, workloads
    from tests._cases import gpu_problem, gpu_quadrature
    o = ipm.default_options("mixed")
    assert (o.precision, o.max_newton, o.max_halvings, o.hessian_reuse, o.newton_kernel, o.check_cache) == (
        ipm.PRECISION["mixed"], 100, 30, 0, 0, 1)
    assert o.newton_tol == 1e-10 and o.reuse_ratio == 0.5
    w = workloads.SOD_1D
    pr, quad = gpu_problem(w), gpu_quadrature(w)
    basis = ipm.ipm_basis(w["p"], w["M"])
    ent = ipm.ipm_entropy(ipm.ENTROPY[w["entropy"]], 0.0, 0.0)
    b = ctypes.c_size_t()
    for bad in (dict(check_cache=2), dict(newton_kernel=3), dict(hessian_reuse=3)):
        ob = ipm.default_options("fp64", **bad)
        st = libipm.ipm_footprint(ctypes.byref(pr), ctypes.byref(basis), ctypes.byref(quad), ctypes.byref(ent),
                                  ctypes.byref(ob), ctypes.byref(b))
        assert st == 1, (bad, st)


def test_noalloc_rejects_unknown_kinds_before_device_work(libipm):
    """ipm_dual_solve_noalloc validates the problem and entropy kinds before touching the device: an
    unknown entropy kind on an Euler problem, or an unknown problem kind, is IPM_EINVAL (the buffer
    arguments are never dereferenced on this path)."""
    import ctypes
    from paper_1912_09238_gb300 import ipm
    b = ipm.ipm_basis(3, 2)
    q = ipm.ipm_quadrature(n_per_dim=3)
    o = ipm.default_options("fp64")
    s = ipm.ipm_stats()
    fake = ctypes.c_void_p(256)          # never dereferenced: the call returns during validation
    for kind, ent in ((ipm.PROBLEM["euler1d"], 7), (ipm.PROBLEM["euler1d"], -1), (ipm.PROBLEM["euler2d"], 2), (9, 2)):
        e = ipm.ipm_entropy(ent, 0.0, 0.0)
        st = libipm.ipm_dual_solve_noalloc(kind, 1.4, ctypes.byref(b), ctypes.byref(q), ctypes.byref(e),
                                           ctypes.byref(o), 4, fake, fake, fake, fake, fake, None, ctypes.byref(s))
        assert st == 1, (kind, ent, st)
        assert b"kind" in libipm.ipm_last_error(None)
