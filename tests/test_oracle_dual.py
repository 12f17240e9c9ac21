"""Pins of oracle.dual: the dual cost L (Eq. L), its gradient and Hessian (Sec. 3.1), the Newton map
(Eq. dualIterationFunction) and the round trip u_hat = h(lambda_hat) (Eq. ulambda)."""
import numpy as np
import pytest

from oracle import basis, dual, entropy


def manufactured_euler(rng, C, dim, p, M, nq, amp=0.15):
    """Dual states lambda* = projection of grad s of smooth admissible nodal fields."""
    sp = basis.StochasticSpace(p, M, nq)
    ent = entropy.Euler(1.4, dim)
    rho = rng.uniform(0.2, 2.0, (C, 1)) * (1 + amp * np.tanh(sp.nodes @ rng.normal(size=(p, C))).T)
    vel = rng.uniform(-1.0, 1.0, (C, 1, dim)) * (1 + amp * np.sin(sp.nodes @ rng.normal(size=(p, dim)))[None])
    pr = rng.uniform(0.1, 2.0, (C, 1)) * (1 + amp * np.cos(sp.nodes @ rng.normal(size=(p, C))).T)
    u = ent.conserved(rho, vel, pr)
    lam_star = sp.project(ent.grad_s(u))
    return sp, ent, lam_star


def test_gradient_is_derivative_of_cost(rng):
    sp, ent, lam = manufactured_euler(rng, 4, 1, 2, 3, 4)
    uhat = dual.moments_from_duals(sp, ent, lam) * 1.01
    g = dual.dual_gradient(sp, ent, lam, uhat)
    h = 1e-6
    for (i, a) in [(0, 0), (1, 2), (5, 1), (9, 0)]:
        e = np.zeros_like(lam)
        e[:, i, a] = h
        fd = (dual.dual_cost(sp, ent, lam + e, uhat)[0] - dual.dual_cost(sp, ent, lam - e, uhat)[0]) / (2 * h)
        np.testing.assert_allclose(fd, g[:, i, a], rtol=1e-6, atol=1e-7)


def test_hessian_is_derivative_of_gradient(rng):
    sp, ent, lam = manufactured_euler(rng, 3, 2, 2, 2, 3)
    uhat = np.zeros_like(lam)
    H = dual.dual_hessian(sp, ent, lam)
    m = ent.m
    h = 1e-6
    for (j, b) in [(0, 0), (2, 3), (4, 1), (5, 2)]:
        e = np.zeros_like(lam)
        e[:, j, b] = h
        fd = (dual.dual_gradient(sp, ent, lam + e, uhat) - dual.dual_gradient(sp, ent, lam - e, uhat)) / (2 * h)
        np.testing.assert_allclose(fd.reshape(3, -1), H[:, :, j * m + b], rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(H, np.swapaxes(H, 1, 2), rtol=1e-12, atol=1e-13)
    assert np.all(np.linalg.eigvalsh(H) > 0)


@pytest.mark.parametrize("dim,p,M,nq", [(1, 3, 2, 3), (1, 3, 5, 6), (2, 2, 4, 5), (1, 1, 5, 10)])
def test_round_trip_recovers_moments(rng, dim, p, M, nq):
    C = 6 if M < 5 else 3
    sp, ent, lam_star = manufactured_euler(rng, C, dim, p, M, nq)
    uhat = dual.moments_from_duals(sp, ent, lam_star)
    lam0 = np.zeros_like(lam_star)
    lam0[:, 0, :] = lam_star[:, 0, :]            # mean only: a far start
    lam, it, st, res = dual.dual_solve(sp, ent, lam0, uhat, dual.NewtonOptions(tau=1e-13))
    assert np.all(st == dual.OK), st
    assert np.all(res < 1e-13)
    back = dual.moments_from_duals(sp, ent, lam)
    rel = np.max(np.abs(back - uhat)) / np.max(np.abs(uhat))
    assert rel < 1e-12
    np.testing.assert_allclose(lam, lam_star, rtol=1e-8, atol=1e-8)


def test_barrier_round_trip(rng):
    sp = basis.StochasticSpace(1, 5, 10)
    ent = entropy.BoundedBarrier(0.5, 13.0)
    u = 0.5 + 12.5 / (1 + np.exp(-(rng.normal(size=(8, 1)) + 2 * np.tanh(3 * sp.nodes[:, 0])[None])))
    lam_star = sp.project(ent.grad_s(u[..., None]))
    uhat = dual.moments_from_duals(sp, ent, lam_star)
    lam0 = np.zeros_like(lam_star)
    lam, it, st, res = dual.dual_solve(sp, ent, lam0, uhat, dual.NewtonOptions(tau=1e-13))
    assert np.all(st == 0)
    back = dual.moments_from_duals(sp, ent, lam)
    assert np.max(np.abs(back - uhat)) / np.max(np.abs(uhat)) < 1e-12


def test_quadratic_entropy_is_one_newton_step(rng):
    """Quadratic entropy: u_s = Lambda, H = Phi^T W Phi = I (exact quadrature), so lambda_hat = u_hat
    after exactly one step from any start (the SG special case, Sec. 1 and Sec. 3.1)."""
    sp = basis.StochasticSpace(2, 4, 5)
    ent = entropy.Quadratic(4)
    uhat = rng.normal(size=(5, sp.N, 4))
    lam0 = rng.normal(size=(5, sp.N, 4))
    lam, it, st, res = dual.dual_solve(sp, ent, lam0, uhat)
    assert np.all(st == 0) and np.all(it == 1)
    np.testing.assert_allclose(lam, uhat, rtol=1e-13, atol=1e-13)


def test_stopping_criterion_and_cap(rng):
    sp, ent, lam_star = manufactured_euler(rng, 4, 1, 3, 2, 3)
    uhat = dual.moments_from_duals(sp, ent, lam_star)
    lam0 = np.zeros_like(lam_star)
    lam0[:, 0] = lam_star[:, 0]
    _, it, st, res = dual.dual_solve(sp, ent, lam0, uhat, dual.NewtonOptions(tau=1e-10))
    assert np.all(res < 1e-10) and np.all(st == 0)
    _, it1, st1, _ = dual.dual_solve(sp, ent, lam0, uhat, dual.NewtonOptions(tau=1e-10, max_iter=1))
    assert np.all(st1 == dual.NOCONV) and np.all(it1 == 1)


def test_infeasible_start_is_reported():
    sp = basis.StochasticSpace(1, 2, 3)
    ent = entropy.Euler(1.4, 1)
    lam = np.zeros((1, sp.N, 3))
    lam[0, 0, 2] = +1.0                        # Lambda_E > 0 everywhere: u_s undefined
    _, _, st, _ = dual.dual_solve(sp, ent, lam, np.ones((1, sp.N, 3)))
    assert st[0] == dual.INFEASIBLE
