"""Pins of oracle.entropy: the IPM ansatz u_s = (grad s)^-1 (Sec. 3.1), s_* (Sec. 2, Eq. dualProblem),
grad u_s, and the App. B Euler formulas (with the two garble readings)."""
import numpy as np
import pytest

from oracle import entropy


def random_euler_states(rng, n, dim):
    rho = rng.uniform(0.1, 3.0, n)
    vel = rng.uniform(-2.0, 2.0, (n, dim))
    p = rng.uniform(0.05, 3.0, n)
    return entropy.Euler(1.4, dim).conserved(rho, vel, p)


def entropies(rng):
    out = []
    for dim in (1, 2):
        e = entropy.Euler(1.4, dim)
        out.append((e, random_euler_states(rng, 64, dim)))
    b = entropy.BoundedBarrier(0.5, 13.0)
    out.append((b, rng.uniform(0.6, 12.9, (64, 1))))
    q = entropy.Quadratic(3)
    out.append((q, rng.normal(size=(64, 3))))
    return out


def test_round_trip_u_to_lambda_to_u(rng):
    for ent, u in entropies(rng):
        Lam = ent.grad_s(u)
        np.testing.assert_allclose(ent.u_s(Lam), u, rtol=1e-12, atol=1e-12, err_msg=ent.name)
        # and back: grad s(u_s(Lam)) = Lam
        np.testing.assert_allclose(ent.grad_s(ent.u_s(Lam)), Lam, rtol=1e-11, atol=1e-11, err_msg=ent.name)


def test_grad_s_by_finite_differences(rng):
    for ent, u in entropies(rng):
        h = 1e-6
        g = ent.grad_s(u)
        for a in range(ent.m):
            e = np.zeros(ent.m)
            e[a] = h
            fd = (ent.s(u + e) - ent.s(u - e)) / (2 * h)
            np.testing.assert_allclose(fd, g[:, a], rtol=1e-7, atol=1e-7, err_msg=ent.name)


def test_hess_s_by_finite_differences(rng):
    for ent, u in entropies(rng):
        h = 1e-6
        Hs = ent.hess_s(u)
        for a in range(ent.m):
            e = np.zeros(ent.m)
            e[a] = h
            fd = (ent.grad_s(u + e) - ent.grad_s(u - e)) / (2 * h)
            np.testing.assert_allclose(fd, Hs[:, :, a], rtol=1e-6, atol=1e-6, err_msg=ent.name)


def test_s_star_gradient_is_u_s(rng):
    # grad s_* = u_s (Sec. 3.1, below the gradient of L)
    for ent, u in entropies(rng):
        Lam = ent.grad_s(u)
        h = 1e-6
        for a in range(ent.m):
            e = np.zeros(ent.m)
            e[a] = h
            fd = (ent.s_star(Lam + e) - ent.s_star(Lam - e)) / (2 * h)
            np.testing.assert_allclose(fd, u[:, a], rtol=1e-6, atol=1e-6, err_msg=ent.name)


def test_du_s_is_jacobian_and_spd(rng):
    for ent, u in entropies(rng):
        Lam = ent.grad_s(u)
        J = ent.du_s(Lam)
        np.testing.assert_allclose(J, np.swapaxes(J, -1, -2), rtol=1e-10, atol=1e-12)
        assert np.all(np.linalg.eigvalsh(J) > 0)
        h = 1e-6
        for a in range(ent.m):
            e = np.zeros(ent.m)
            e[a] = h
            fd = (ent.u_s(Lam + e) - ent.u_s(Lam - e)) / (2 * h)
            np.testing.assert_allclose(fd, J[:, :, a], rtol=1e-6, atol=1e-6, err_msg=ent.name)


@pytest.mark.parametrize("dim", [1, 2])
def test_euler_s_star_is_gamma_minus_one_rho(rng, dim):
    ent = entropy.Euler(1.4, dim)
    u = random_euler_states(rng, 50, dim)
    Lam = ent.grad_s(u)
    np.testing.assert_allclose(ent.s_star(Lam), 0.4 * u[:, 0], rtol=1e-12, atol=1e-13)


def test_euler_printed_alpha_exponent_fails_round_trip():
    """The exponent printed in App. B (-2 Lambda_4 gamma) does not invert grad s; the reading with
    +2 gamma Lambda_4 does. The example state is the one named when the reading was adopted."""
    g = 1.4
    ent = entropy.Euler(g, 2)
    u = np.array([[1.3, 0.4, -0.2, 2.5]])
    Lam = ent.grad_s(u)
    L1, L2, L3, L4 = Lam[0]
    printed = np.exp((L2 ** 2 + L3 ** 2 - 2 * L1 * L4 - 2 * L4 * g) / (2 * L4 * (1 - g))) * (-L4) ** (1 / (1 - g))
    assert abs(printed - 1.3) > 1.0
    np.testing.assert_allclose(ent.u_s(Lam)[0], u[0], rtol=1e-13)


def test_euler_app_b_gradient_components():
    # dS/dE = -rho / (E - |m|^2/(2 rho)); dS/dm_i = m_i / (E - |m|^2/(2 rho)) (App. B, m_i printed form)
    ent = entropy.Euler(1.4, 2)
    u = np.array([[0.7, 0.3, 0.1, 1.9]])
    rho, m1, m2, E = u[0]
    eps = E - (m1 ** 2 + m2 ** 2) / (2 * rho)
    g = ent.grad_s(u)[0]
    assert abs(g[3] + rho / eps) < 1e-14
    assert abs(g[1] - m1 / eps) < 1e-14 and abs(g[2] - m2 / eps) < 1e-14


def test_barrier_closed_forms():
    ent = entropy.BoundedBarrier(0.5, 13.0)
    D = 12.5
    Lam = np.linspace(-30, 30, 61)[:, None]
    u = ent.u_s(Lam)[:, 0]
    assert np.all(u > 0.5) and np.all(u < 13.0)
    np.testing.assert_allclose(ent.u_s(np.zeros((1, 1)))[0, 0], 6.75, rtol=1e-15)
    # s_*(Lambda) = D ln(1 + e^Lambda) + u_- Lambda - D ln D
    ref = D * np.logaddexp(0.0, Lam[:, 0]) + 0.5 * Lam[:, 0] - D * np.log(D)
    mid = np.abs(Lam[:, 0]) < 25      # away from the saturated tails where Lambda u - s(u) cancels
    np.testing.assert_allclose(ent.s_star(Lam)[mid], ref[mid], rtol=1e-10, atol=1e-9)
    # u_s' = (u - u_-)(u_+ - u)/(u_+ - u_-)
    J = ent.du_s(Lam)[:, 0, 0]
    np.testing.assert_allclose(J, (u - 0.5) * (13.0 - u) / D, rtol=1e-9, atol=1e-300)


def test_euler_feasibility():
    ent = entropy.Euler(1.4, 1)
    Lam = np.array([[0.1, 0.2, -0.5], [0.1, 0.2, 0.0], [0.1, 0.2, 0.3]])
    assert list(ent.feasible(Lam)) == [True, False, False]
