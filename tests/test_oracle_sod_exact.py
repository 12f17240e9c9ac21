"""Pin of the oracle's Euler path against the exact Riemann solution (no GPU).

The uncertain Sod tube (rho_L = 1 + 0.1 xi_1, p_L = 1 + 0.1 xi_2, interface 0.5 + 0.05 xi_3, right state
(0.125, 0, 0.1), gamma = 1.4) has, for every xi, an exact self-similar solution: a left rarefaction, a
contact and a right shock. tests/_riemann.py builds it from the wave relations (independent of oracle/)
and collocates it by brute force over xi. The IPM scheme of Sec. 3.1 (Algorithm 1 with the Lax-Friedrichs
flux of App. A, Euler entropy of App. B) is first order in space, so its expectation converges to the exact
one only as the mesh is refined; the bounds below are set by the measured refinement sweep (relative L1
errors of E[rho]: 5.6e-2, 4.2e-2, 3.1e-2 at 50, 100, 200 cells; 2.2e-2 at 400), with margin. A wrong flux,
entropy, initial projection or time step moves these errors far outside the bounds or stops their decrease.
"""
import numpy as np
import pytest

from paper_1912_09238_gb300 import workloads
from tests._cases import oracle_problem
from tests._riemann import RiemannSolution, sod_density_moments

GAMMA = 1.4


def _cons(rho, u, p):
    return rho, rho * u, p / (GAMMA - 1.0) + 0.5 * rho * u * u


@pytest.mark.parametrize("left,right", [((1.0, 0.0, 1.0), (0.125, 0.0, 0.1)),        # Sod
                                        ((1.1, 0.0, 0.9), (0.125, 0.0, 0.1)),        # a perturbed Sod
                                        ((0.125, 0.0, 0.1), (1.0, 0.0, 1.0))])       # mirrored
def test_exact_solution_satisfies_the_wave_relations(left, right):
    """Rankine-Hugoniot conditions across the shock (mass, momentum and energy fluxes in the shock frame),
    the isentropic relation and the Riemann invariant across the rarefaction, continuity at the edges of
    the fan, and the mirror symmetry of the solution."""
    sol = RiemannSolution(left, right, GAMMA)
    shock = 1 if sol.ps > right[2] else -1
    fan = -shock
    # shock: [rho (u - S)] = [rho u (u - S) + p] = [E (u - S) + p u] = 0
    S = sol.shock_speed(shock)
    Wo = right if shock > 0 else left
    ro, mo, Eo = _cons(*Wo)
    rs, ms, Es = _cons(sol.star_density(shock), sol.us, sol.ps)
    for a, b in ((rs * (sol.us - S), ro * (Wo[1] - S)),
                 (ms * (sol.us - S) + sol.ps, mo * (Wo[1] - S) + Wo[2]),
                 (Es * (sol.us - S) + sol.ps * sol.us, Eo * (Wo[1] - S) + Wo[2] * Wo[1])):
        assert abs(a - b) <= 1e-12 * max(abs(a), abs(b), 1.0)
    # rarefaction: p / rho^gamma and u -+ 2c/(gamma-1) are carried across it
    Wf = left if fan < 0 else right
    rf = sol.star_density(fan)
    assert abs(sol.ps / rf ** GAMMA - Wf[2] / Wf[0] ** GAMMA) <= 1e-12 * Wf[2] / Wf[0] ** GAMMA
    cf, c0 = np.sqrt(GAMMA * sol.ps / rf), np.sqrt(GAMMA * Wf[2] / Wf[0])
    sign = 1.0 if fan < 0 else -1.0
    assert abs((sol.us + sign * 2 * cf / (GAMMA - 1)) - (Wf[1] + sign * 2 * c0 / (GAMMA - 1))) <= 1e-12
    # the sampled profile is continuous at the head and the tail of the fan
    head = Wf[1] + fan * c0
    tail = sol.us + fan * cf
    for edge, inner in ((head, Wf[0]), (tail, rf)):
        r, _, _ = sol.sample(np.array([edge - 1e-9, edge + 1e-9]))
        assert np.abs(r - inner).max() < 1e-6
    # mirror: rho(s) of the mirrored problem equals rho(-s)
    mir = RiemannSolution((right[0], -right[1], right[2]), (left[0], -left[1], left[2]), GAMMA)
    s = np.linspace(-2.0, 2.0, 401) + 1e-7
    assert np.abs(sol.sample(s)[0] - mir.sample(-s)[0]).max() < 1e-9


def test_sod_star_state():
    """The classic Sod star state (p* = 0.30313, u* = 0.92745 to the five digits usually quoted)."""
    sol = RiemannSolution((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), GAMMA)
    assert abs(sol.ps - 0.30313) < 5e-6 and abs(sol.us - 0.92745) < 5e-6


def test_ipm_expectation_converges_to_the_exact_collocation():
    """Algorithm 1 of the oracle (total degree 2 in 3 dims, 3^3 Gauss nodes) to t_end = 0.14 on 50, 100 and
    200 cells: the relative L1 errors of E[rho] and Var[rho] against the brute-force collocation of the exact
    solution fall under refinement and stay within the measured bounds."""
    from oracle import scheme1d as s1
    errs_e, errs_v = [], []
    for nx in (50, 100, 200):
        w = workloads.variant(workloads.SOD_1D, nx=nx, M=2, nq=3)
        st = s1.run(oracle_problem(w))
        assert abs(st.t - 0.14) < 1e-12
        E = st.uhat[1:-1, 0, 0]
        V = np.sum(st.uhat[1:-1, 1:, 0] ** 2, axis=1)
        Er, Vr = sod_density_moments(nx, 0.0, 1.0, st.t, GAMMA)
        errs_e.append(np.abs(E - Er).sum() / np.abs(Er).sum())
        errs_v.append(np.abs(V - Vr).sum() / np.abs(Vr).sum())
    assert errs_e[0] < 0.065 and errs_e[1] < 0.048 and errs_e[2] < 0.035, errs_e
    assert errs_e[1] < 0.85 * errs_e[0] and errs_e[2] < 0.85 * errs_e[1], errs_e
    assert errs_v[2] < errs_v[1] < errs_v[0] < 0.55, errs_v
