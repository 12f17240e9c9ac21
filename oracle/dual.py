"""The IPM dual problem and its Newton solver (test infrastructure; see ``oracle/__init__``).

For one cell with moments u_hat in R^{N x m} (Sec. 3.1):
* cost       L(lambda; u_hat) = <s_*(lambda^T phi)>_Q - sum_i lambda_i . u_hat_i           (Eq. L)
* gradient   grad L = <u_s(lambda^T phi) phi^T>_Q^T - u_hat                                 (Sec. 3.1)
* Hessian    H = <grad u_s(lambda^T phi) (x) phi phi^T>_Q, entry ((i,a),(j,b)) =
             sum_k w_k [grad u_s]_{ab}(Lambda_k) phi_i(xi_k) phi_j(xi_k); flat index i*m + a
* Newton map d(lambda, u_hat) = lambda - H^-1 grad L                         (Eq. dualIterationFunction)
* stop when  sum_i || grad_{lambda_i} L ||_2 < tau                                         (Eq. tauCrit;
             the printed index range is garbled: the sum runs over the N multi-indices i).

Line search (not in the paper, which takes full Newton steps): Armijo backtracking on L. The step
is alpha * Delta with Delta = -H^-1 grad L, alpha = 1, 1/2, 1/4, ... (at most ``max_halvings``
halvings). A trial is accepted when every node is feasible (u_s defined and finite) and
    L(lambda + alpha Delta) <= L(lambda) + c alpha (grad L . Delta) + slack,
    slack = slack_rel * (1 + sum_k w_k |s_*(Lambda_k)| + sum_{i,a} |lambda_ia u_hat_ia|),
where the slack absorbs the rounding of L near the minimiser (there the true decrease falls
below the rounding of L). Near the solution the full step is taken, so the fixed point and the
quadratic convergence of Newton's method are unchanged.

Per-cell status codes: 0 converged, 1 iteration cap reached, 2 line search failed,
3 infeasible starting point, 4 non-finite gradient / singular Hessian.

Pinned by: tests/test_oracle_dual.py (round trip u_hat = h(lambda*) recovered to 1e-12; quadratic
entropy converges in one step with lambda = u_hat; finite-difference gradient and Hessian of L).
"""
from dataclasses import dataclass

import numpy as np

OK, NOCONV, LINESEARCH, INFEASIBLE, NONFINITE = 0, 1, 2, 3, 4


@dataclass
class NewtonOptions:
    tau: float = 1e-10
    max_iter: int = 100
    armijo_c: float = 1e-4
    max_halvings: int = 30
    slack_rel: float = 1e-12


def reconstruct(space, lam):
    """Lambda_k = lambda^T phi(xi_k) at every node: (C, N, m) -> (C, Q, m)."""
    return space.evaluate(lam)


def dual_cost(space, ent, lam, uhat):
    """L(lambda; u_hat) per cell (Eq. L). Returns (L, scale) with scale the slack magnitude."""
    Lam = reconstruct(space, lam)
    sst = ent.s_star(Lam)                                   # (C, Q)
    lin = np.sum(lam * uhat, axis=(-2, -1))
    L = sst @ space.w - lin
    scale = np.abs(sst) @ space.w + np.sum(np.abs(lam * uhat), axis=(-2, -1))
    return L, scale


def dual_gradient(space, ent, lam, uhat):
    """grad L = <u_s(lambda^T phi) phi^T>_Q^T - u_hat, shape (C, N, m)."""
    return space.project(ent.u_s(reconstruct(space, lam))) - uhat


def dual_hessian(space, ent, lam):
    """H((i,a),(j,b)) = <[grad u_s]_ab phi_i phi_j>_Q, flattened to (C, N*m, N*m) with index i*m+a."""
    J = ent.du_s(reconstruct(space, lam))                   # (C, Q, m, m)
    C = lam.shape[0]
    N, m = space.N, ent.m
    H = np.einsum("k,ckab,ki,kj->ciajb", space.w, J, space.Phi, space.Phi, optimize=True)
    return H.reshape(C, N * m, N * m)


def residual_norm(g):
    """sum over multi-indices i of the Euclidean norm of grad_{lambda_i} L (Eq. tauCrit)."""
    return np.sum(np.sqrt(np.sum(g * g, axis=-1)), axis=-1)


def newton_direction(H, g):
    """Delta = -H^-1 grad L (flattened index i*m + a)."""
    C, N, m = g.shape
    return -np.linalg.solve(H, g.reshape(C, N * m)[..., None])[..., 0].reshape(C, N, m)


def _armijo(space, ent, lam, uhat, g, delta, opts):
    """Backtracking on L for a batch of cells. Returns (alpha, accepted) per cell."""
    C = lam.shape[0]
    L0, scale = dual_cost(space, ent, lam, uhat)
    slope = np.sum(g * delta, axis=(-2, -1))
    slack = opts.slack_rel * (1.0 + scale)
    alpha = np.ones(C)
    accepted = np.zeros(C, dtype=bool)
    for _ in range(opts.max_halvings + 1):
        todo = ~accepted
        if not np.any(todo):
            break
        idx = np.nonzero(todo)[0]
        lt = lam[idx] + alpha[idx, None, None] * delta[idx]
        feas = np.all(ent.feasible(reconstruct(space, lt)), axis=-1)
        with np.errstate(invalid="ignore", over="ignore", divide="ignore"):
            Lt, _ = dual_cost(space, ent, lt, uhat[idx])
            ok = feas & np.isfinite(Lt) & (Lt <= L0[idx] + opts.armijo_c * alpha[idx] * slope[idx] + slack[idx])
        accepted[idx[ok]] = True
        still = idx[~ok]
        alpha[still] *= 0.5
    return alpha, accepted


def dual_solve(space, ent, lam0, uhat, opts: NewtonOptions = NewtonOptions(), one_step: bool = False):
    """Newton iteration (Eq. dualIteration1) per cell, warm-started at lam0.

    one_step=False: iterate until Eq. tauCrit holds (Algorithm 1, inner loop).
    one_step=True : apply the (damped) Newton map d exactly once (Algorithm 2, Eq. oneshotIPMdual).
    Returns (lam, iterations, status, residual) with residual the criterion at the last gradient.
    """
    lam = np.array(lam0, dtype=np.float64, copy=True)
    C = lam.shape[0]
    iters = np.zeros(C, dtype=np.int64)
    status = np.zeros(C, dtype=np.int64)
    resid = np.full(C, np.inf)
    active = np.ones(C, dtype=bool)

    start_ok = np.all(ent.feasible(reconstruct(space, lam)), axis=-1)
    status[~start_ok] = INFEASIBLE
    active &= start_ok

    max_iter = 1 if one_step else opts.max_iter
    for it in range(max_iter + 1):
        idx = np.nonzero(active)[0]
        if idx.size == 0:
            break
        with np.errstate(invalid="ignore", over="ignore"):
            g = dual_gradient(space, ent, lam[idx], uhat[idx])
        r = residual_norm(g)
        resid[idx] = r
        bad = ~np.isfinite(r)
        status[idx[bad]] = NONFINITE
        active[idx[bad]] = False
        if one_step:
            if it == 1:
                break
            go = ~bad
        else:
            conv = (r < opts.tau) & ~bad
            active[idx[conv]] = False
            if it == max_iter:
                left = idx[~conv & ~bad]
                status[left] = NOCONV
                active[left] = False
                break
            go = ~conv & ~bad
        sel = idx[go]
        if sel.size == 0:
            continue
        gs = g[go]
        H = dual_hessian(space, ent, lam[sel])
        try:
            delta = newton_direction(H, gs)
        except np.linalg.LinAlgError:
            # fall back to one cell at a time to find the singular ones
            delta = np.zeros_like(gs)
            for t, c in enumerate(sel):
                try:
                    delta[t] = newton_direction(H[t:t + 1], gs[t:t + 1])[0]
                except np.linalg.LinAlgError:
                    status[c] = NONFINITE
                    active[c] = False
        alpha, acc = _armijo(space, ent, lam[sel], uhat[sel], gs, delta, opts)
        acc &= active[sel]
        lam[sel[acc]] += alpha[acc, None, None] * delta[acc]
        iters[sel[acc]] += 1
        fail = sel[~acc & active[sel]]
        status[fail] = LINESEARCH
        active[fail] = False
    return lam, iters, status, resid


def moments_from_duals(space, ent, lam):
    """h(lambda) = <u_s(lambda^T phi) phi^T>_Q^T (Sec. 4, Eq. ulambda, with the quadrature)."""
    return space.project(ent.u_s(reconstruct(space, lam)))
