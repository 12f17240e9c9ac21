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


def test_retardation_caps_levels_then_releases_them():
    """Algorithm 4 on a coarse ramp: the cap holds every level at the coarsest degree until the residual
    passes the stage tolerance; afterwards finer levels appear; the residual keeps falling."""
    w = workloads.variant(workloads.RAMP_2D, nx=10, ny=5, M=4, nq=5, sides=("dirichlet", "outflow", "slip", "dirichlet"))
    prob = oracle_problem_2d(w)
    lv = ad.Levels(degrees=(2, 3, 4), delta_lo=1e-10, delta_hi=1e-8)
    st, hist = ad.oneshot_retarded(prob, lv, caps=(0, 2), tolerances=(2e-3,), tol=1e-9, max_steps=60)
    stages = [h[2] for h in hist]
    assert stages[0] == 0 and stages[-1] == 1
    first1 = stages.index(1)
    assert hist[first1 - 1][1] < 2e-3 <= max(h[1] for h in hist[:first1 - 1] or [(0, 1.0, 0)])
    assert st.level[1:-1, 1:-1].max() > 0                   # finer degrees once released
    assert hist[-1][1] < hist[0][1]


def test_oneshot_step_with_cap_zero_is_the_fixed_low_degree_oneshot():
    w = workloads.variant(workloads.RAMP_2D, nx=8, ny=4, M=4, nq=5)
    prob = oracle_problem_2d(w)
    lv = ad.Levels(degrees=(2, 3, 4), delta_lo=2e-5, delta_hi=2e-4)
    nl, _ = ad.level_sizes(prob.space, lv)
    a = ad.cap_levels(ad.initial_state(prob, lv), 0, nl)
    w2 = workloads.variant(w, M=2)
    prob2 = oracle_problem_2d(w2)
    f = s2.initial_state(prob2)
    assert np.abs(a.uhat[..., :nl[0], :] - f.uhat).max() < 1e-14
    for _ in range(3):
        a = ad.oneshot_step(prob, a, lv, 0)
        f = s2.oneshot_step(prob2, f)
        assert np.abs(a.uhat[..., :nl[0], :] - f.uhat).max() < 1e-12
        assert np.all(a.uhat[..., nl[0]:, :] == 0.0)


# ---------- quadrature per refinement level (nested Clenshaw-Curtis rules, Sec. 5 and Sec. 7) ----------
def _kh_cc(nx=8, M=2, kmax=3, p=2):
    """The shear layer with two uncertain dims (band half-width 0.25 + 0.05 xi_1, phase 0.1 xi_2) in a
    nested Clenshaw-Curtis space of level kmax."""
    w = workloads.variant(workloads.KH_2D, nx=nx, ny=nx, M=M, nq=3, dparam=((0.005, 0.0, 0.0), (0.0, 0.1, 0.0),
                                                                          (0.05, 0.0, 0.0), (0.0, 0.0, 0.0)), p=p)
    prob = oracle_problem_2d(w)
    prob.space = basis.NestedCCSpace(p, M, kmax)
    return w, prob


def test_single_level_with_its_own_rule_is_the_fixed_rule_scheme():
    """One refinement level on the level-2 rule, inside a level-3 nested space, equals the fixed-degree
    scheme whose space is the level-2 rule itself."""
    _, prob = _kh_cc(kmax=3)
    lv = ad.Levels(degrees=(2,), delta_lo=2e-5, delta_hi=2e-4, quad_levels=(2,))
    _, ref = _kh_cc(kmax=2)
    a = ad.initial_state(prob, lv)
    f = s2.initial_state(ref)
    assert np.abs(a.uhat - f.uhat).max() < 1e-14
    for _ in range(2):
        a = ad.ipm_step(prob, a, lv)
        f = s2.ipm_step(ref, f)
        assert np.abs(a.uhat - f.uhat).max() < 1e-12
        assert abs(a.last_dt - f.last_dt) <= 1e-15 * f.last_dt


def test_levels_sharing_one_rule_equal_the_shared_rule_scheme():
    """Two refinement levels that both use the finest rule of the space give the shared-rule scheme."""
    _, prob = _kh_cc(M=3, kmax=2)
    lv_q = ad.Levels(degrees=(2, 3), delta_lo=2e-5, delta_hi=2e-4, quad_levels=(2, 2))
    lv_s = ad.Levels(degrees=(2, 3), delta_lo=2e-5, delta_hi=2e-4)
    a, b = ad.initial_state(prob, lv_q), ad.initial_state(prob, lv_s)
    assert np.array_equal(a.level, b.level) and np.abs(a.uhat - b.uhat).max() < 1e-14
    for _ in range(2):
        a, b = ad.ipm_step(prob, a, lv_q), ad.ipm_step(prob, b, lv_s)
        assert np.array_equal(a.level, b.level)
        assert np.abs(a.uhat - b.uhat).max() < 1e-12


def test_per_level_rules_change_levels_keep_zeros_and_conserve_within_one_level():
    _, prob = _kh_cc(nx=10, M=3, kmax=2)
    lv = ad.Levels(degrees=(1, 2, 3), delta_lo=2e-5, delta_hi=2e-4, quad_levels=(1, 2, 2))
    nl, _ = ad.level_sizes(prob.space, lv)
    st = ad.initial_state(prob, lv)
    seen = set()
    for _ in range(3):
        st = ad.ipm_step(prob, st, lv)
        assert np.all(st.newton_status == 0)
        lev = st.level[1:-1, 1:-1]
        seen |= set(np.unique(lev).tolist())
        n = np.asarray(nl)[lev]
        beyond = np.arange(st.uhat.shape[-2])[None, None, :] >= n[..., None]
        assert np.all(st.uhat[1:-1, 1:-1][beyond] == 0.0)
    assert len(seen) >= 2
    # every cell on one level (the coarsest, a 3-point rule per dimension): the fluxes telescope and the
    # means are conserved up to the dual residuals
    lv1 = ad.Levels(degrees=(1,), delta_lo=2e-5, delta_hi=2e-4, quad_levels=(1,))
    st = ad.initial_state(prob, lv1)
    A = prob.mesh.area()
    for _ in range(3):
        old = st
        st = ad.ipm_step(prob, old, lv1)
        tot = np.sum(A[..., None] * st.uhat[1:-1, 1:-1, 0, :], axis=(0, 1))
        tot0 = np.sum(A[..., None] * old.uhat[1:-1, 1:-1, 0, :], axis=(0, 1))
        assert np.abs(tot - tot0).max() < 1e-9
