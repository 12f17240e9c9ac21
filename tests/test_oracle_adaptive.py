"""Pins of the adaptive oracle (Algorithm 3, Eq. errorIndicator) in oracle/adaptive.py."""
import numpy as np

from oracle import adaptive as ad
from oracle import basis
from oracle import scheme2d as s2
from paper_1912_09238_gb300 import workloads
from tests._cases import oracle_problem_2d


def test_indicator_equals_its_integral_definition():
    """S_l = <(u_l - u_{l-1})^2>/<u_l^2> computed on the nodes from the truncated expansions equals
    the shell-energy form used by the oracle (orthonormal basis, exact quadrature)."""
    sp = basis.StochasticSpace(3, 4, 5)
    lv = ad.Levels(degrees=(2, 3, 4), delta_lo=2e-4, delta_hi=2e-5)
    nl, nprev = ad.level_sizes(sp, lv)
    assert nl == [10, 20, 35] and nprev == [4, 10, 20]
    rng = np.random.default_rng(5)
    u = rng.standard_normal((7, sp.N)) * np.exp(-0.4 * np.sum(sp.indices, axis=1))
    for l in range(3):
        ul = np.einsum("ki,ci->ck", sp.Phi[:, :nl[l]], u[:, :nl[l]])
        up = np.einsum("ki,ci->ck", sp.Phi[:, :nprev[l]], u[:, :nprev[l]])
        S_int = ((ul - up) ** 2 @ sp.w) / (ul ** 2 @ sp.w)
        assert np.allclose(ad.indicator(u, nl[l], nprev[l]), S_int, rtol=1e-12, atol=0)


def test_level_rules_keep_lower_raise_and_clamp():
    sp = basis.StochasticSpace(1, 4, 5)
    lv = ad.Levels(degrees=(2, 3, 4), delta_lo=2e-4, delta_hi=2e-5)     # printed order; interval [2e-5, 2e-4]
    nl, nprev = ad.level_sizes(sp, lv)                                 # 1-D: N_l = M_l + 1
    def state(top_energy):
        u = np.zeros((1, sp.N, 1))
        u[0, 0, 0] = 1.0
        u[0, 1:, 0] = np.sqrt(top_energy)
        return u
    cases = [(1e-6, 1, 0), (1e-4, 1, 1), (1e-2, 1, 2), (1e-6, 0, 0), (1e-2, 2, 2)]
    for e, lev, want in cases:
        new, S = ad.new_levels(state(e), np.array([lev]), nl, nprev, lv)
        assert new[0] == want, (e, lev, S)


def test_single_level_is_the_fixed_degree_scheme():
    w = workloads.variant(workloads.KH_2D, nx=8, ny=8, M=3, nq=4)
    prob = oracle_problem_2d(w)
    lv = ad.Levels(degrees=(3,), delta_lo=2e-5, delta_hi=2e-4)
    a = ad.initial_state(prob, lv)
    f = s2.initial_state(prob)
    assert np.array_equal(a.uhat, f.uhat) and np.array_equal(a.lam, f.lam)
    for _ in range(2):
        a = ad.ipm_step(prob, a, lv)
        f = s2.ipm_step(prob, f)
        assert np.abs(a.uhat - f.uhat).max() < 1e-13
        assert a.last_dt == f.last_dt


def test_levels_change_and_moments_beyond_the_level_stay_zero_and_means_are_conserved():
    w = workloads.variant(workloads.KH_2D, nx=12, ny=12, M=4, nq=5)
    prob = oracle_problem_2d(w)
    lv = ad.Levels(degrees=(2, 3, 4), delta_lo=2e-4, delta_hi=2e-5)
    nl, _ = ad.level_sizes(prob.space, lv)
    st = ad.initial_state(prob, lv)
    A = prob.mesh.area()
    seen = set()
    for _ in range(4):
        old = st
        st = ad.ipm_step(prob, old, lv)
        assert np.all(st.newton_status == 0)
        lev = st.level[1:-1, 1:-1]
        seen |= set(np.unique(lev).tolist())
        n = np.asarray(nl)[lev]
        idx = np.arange(st.uhat.shape[-2])
        beyond = idx[None, None, :] >= n[..., None]
        assert np.all(st.uhat[1:-1, 1:-1][beyond] == 0.0) and np.all(st.lam[1:-1, 1:-1][beyond] == 0.0)
        # the zero-order moments are never truncated: the means are conserved up to the dual residuals
        tot = np.sum(A[..., None] * st.uhat[1:-1, 1:-1, 0, :], axis=(0, 1))
        tot0 = np.sum(A[..., None] * old.uhat[1:-1, 1:-1, 0, :], axis=(0, 1))
        assert np.abs(tot - tot0).max() < 1e-9
    assert len(seen) >= 2
