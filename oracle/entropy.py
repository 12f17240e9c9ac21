"""Entropies, the IPM ansatz and the dual potential (test infrastructure; see ``oracle/__init__``).

For a strictly convex entropy s : R^m -> R the IPM ansatz is u_s(Lambda) = (grad s)^-1(Lambda)
(Sec. 3.1, definition of u_s; Sec. 2, Eq. ansatz). The dual cost needs the Legendre transform
s_*(Lambda) = Lambda . u - s(u) at u = u_s(Lambda) (Sec. 2, Eq. dualProblem), and Newton needs the
Jacobian grad u_s (Sec. 3.1, the Hessian H).

The oracle computes each object from its plain definition:
* u_s from the closed-form inverse of grad s (App. B for Euler);
* s_* literally as Lambda . u_s(Lambda) - s(u_s(Lambda));
* grad u_s as the matrix inverse of the primal Hessian grad^2 s at u_s(Lambda)
  (inverse-function theorem: u_s = (grad s)^-1 => grad u_s = (grad^2 s)^-1).

Entropies:
* Quadratic  s(u) = |u|^2 / 2: IPM reduces to stochastic Galerkin (Sec. 1; Sec. 3.1).
* BoundedBarrier  s(u) = (u-u_-) ln(u-u_-) + (u_+-u) ln(u_+-u) for scalar Burgers; the entropy of
  the Burgers workload (not printed in the paper: the cited maximum-principle IPM work).
* Euler  s(u) = -rho ln(rho^-gamma (E - |m|^2/(2 rho))) (App. B), for d = 1 (u = (rho, m, E)) or
  d = 2 (u = (rho, m_1, m_2, E)).

Readings of garbled App. B formulas (both checked by the round-trip pin):
* dS/dE is -rho / (E - |m|^2/(2 rho)); the printed form is garbled.
* the alpha exponent numerator is |Lambda_v|^2 - 2 Lambda_1 Lambda_E + 2 gamma Lambda_E (the
  printed "- 2 Lambda_4 gamma" fails grad s(u_s(Lambda)) = Lambda).

Pinned by: tests/test_oracle_entropy.py (round trip grad s(u_s(L)) = L, finite differences of s_*
and u_s, symmetry/positivity of grad u_s, s_* = (gamma-1) rho for Euler, barrier closed forms).
"""
import numpy as np


class Quadratic:
    """s(u) = |u|^2/2: u_s = Lambda, grad u_s = I, s_* = |Lambda|^2/2."""

    name = "quadratic"

    def __init__(self, m: int):
        self.m = m

    def s(self, u):
        return 0.5 * np.sum(u * u, axis=-1)

    def grad_s(self, u):
        return np.array(u, dtype=np.float64, copy=True)

    def hess_s(self, u):
        return np.broadcast_to(np.eye(self.m), u.shape[:-1] + (self.m, self.m)).copy()

    def u_s(self, Lam):
        return np.array(Lam, dtype=np.float64, copy=True)

    def du_s(self, Lam):
        return np.linalg.inv(self.hess_s(self.u_s(Lam)))

    def s_star(self, Lam):
        u = self.u_s(Lam)
        return np.sum(Lam * u, axis=-1) - self.s(u)

    def feasible(self, Lam):
        return np.all(np.isfinite(Lam), axis=-1)


class BoundedBarrier:
    """Scalar bounded-barrier entropy on (u_-, u_+)."""

    name = "bounded_barrier"

    def __init__(self, u_minus: float, u_plus: float):
        self.m = 1
        self.um, self.up = float(u_minus), float(u_plus)

    def s(self, u):
        v = u[..., 0]
        return (v - self.um) * np.log(v - self.um) + (self.up - v) * np.log(self.up - v)

    def grad_s(self, u):
        v = u[..., 0]
        return (np.log(v - self.um) - np.log(self.up - v))[..., None]

    def hess_s(self, u):
        v = u[..., 0]
        return (1.0 / (v - self.um) + 1.0 / (self.up - v))[..., None, None]

    def u_s(self, Lam):
        # grad s(u) = ln((u-u_-)/(u_+-u)) = Lambda  =>  u = (u_- + u_+ e^Lambda) / (1 + e^Lambda)
        L = Lam[..., 0]
        e = np.exp(-np.abs(L))
        sig = np.where(L >= 0, 1.0 / (1.0 + e), e / (1.0 + e))   # logistic(L), overflow-safe
        return (self.um + (self.up - self.um) * sig)[..., None]

    def du_s(self, Lam):
        return 1.0 / self.hess_s(self.u_s(Lam))

    def s_star(self, Lam):
        u = self.u_s(Lam)
        return Lam[..., 0] * u[..., 0] - self.s(u)

    def feasible(self, Lam):
        return np.all(np.isfinite(Lam), axis=-1)


class Euler:
    """Euler entropy of App. B in d = 1 or 2 space dimensions (m = d + 2)."""

    name = "euler"

    def __init__(self, gamma: float, dim: int):
        self.gamma = float(gamma)
        self.d = dim
        self.m = dim + 2

    def _split(self, u):
        rho = u[..., 0]
        mom = u[..., 1:1 + self.d]
        E = u[..., self.d + 1]
        return rho, mom, E

    def s(self, u):
        rho, mom, E = self._split(u)
        eps = E - np.sum(mom * mom, axis=-1) / (2.0 * rho)
        return -rho * np.log(rho ** (-self.gamma) * eps)

    def grad_s(self, u):
        """App. B gradient (with the corrected dS/dE)."""
        g = self.gamma
        rho, mom, E = self._split(u)
        msq = np.sum(mom * mom, axis=-1)
        eps = E - msq / (2.0 * rho)
        out = np.empty(u.shape, dtype=np.float64)
        out[..., 0] = -np.log(rho ** (-g) * eps) + msq / (-2.0 * rho * E + msq) + g
        out[..., 1:1 + self.d] = -2.0 * rho[..., None] * mom / (-2.0 * rho * E + msq)[..., None]
        out[..., self.d + 1] = -rho / eps
        return out

    def hess_s(self, u):
        """Second derivatives of s, differentiated by hand from the App. B gradient.

        With eps = E - q, q = |m|^2/(2 rho):
          s_rr = gamma/rho + q^2/(rho eps^2); s_rm = -q m/(rho eps^2); s_rE = -1/eps + q/eps^2;
          s_mm = I/eps + m m^T/(rho eps^2);  s_mE = -m/eps^2;         s_EE = rho/eps^2.
        """
        g = self.gamma
        rho, mom, E = self._split(u)
        q = np.sum(mom * mom, axis=-1) / (2.0 * rho)
        eps = E - q
        d, m = self.d, self.m
        Hs = np.zeros(u.shape[:-1] + (m, m))
        Hs[..., 0, 0] = g / rho + q * q / (rho * eps * eps)
        for i in range(d):
            v = -q * mom[..., i] / (rho * eps * eps)
            Hs[..., 0, 1 + i] = v
            Hs[..., 1 + i, 0] = v
            for j in range(d):
                Hs[..., 1 + i, 1 + j] = (1.0 / eps if i == j else 0.0) + mom[..., i] * mom[..., j] / (rho * eps * eps)
            w = -mom[..., i] / (eps * eps)
            Hs[..., 1 + i, d + 1] = w
            Hs[..., d + 1, 1 + i] = w
        Hs[..., 0, d + 1] = -1.0 / eps + q / (eps * eps)
        Hs[..., d + 1, 0] = Hs[..., 0, d + 1]
        Hs[..., d + 1, d + 1] = rho / (eps * eps)
        return Hs

    def u_s(self, Lam):
        """App. B ansatz with the corrected alpha exponent (Lambda_E = last entry < 0)."""
        g = self.gamma
        L1 = Lam[..., 0]
        Lv = Lam[..., 1:1 + self.d]
        LE = Lam[..., self.d + 1]
        lvsq = np.sum(Lv * Lv, axis=-1)
        with np.errstate(invalid="ignore", divide="ignore", over="ignore"):
            alpha = np.exp((lvsq - 2.0 * L1 * LE + 2.0 * g * LE) / (2.0 * LE * (1.0 - g))) * (-LE) ** (1.0 / (1.0 - g))
            out = np.empty(Lam.shape, dtype=np.float64)
            out[..., 0] = alpha
            out[..., 1:1 + self.d] = -Lv * (alpha / LE)[..., None]
            out[..., self.d + 1] = -alpha * (-lvsq + 2.0 * LE) / (2.0 * LE * LE)
        return out

    def du_s(self, Lam):
        return np.linalg.inv(self.hess_s(self.u_s(Lam)))

    def s_star(self, Lam):
        u = self.u_s(Lam)
        with np.errstate(invalid="ignore", divide="ignore", over="ignore"):
            return np.sum(Lam * u, axis=-1) - self.s(u)

    def feasible(self, Lam):
        """u_s is defined iff Lambda_E < 0; also reject non-finite states."""
        LE = Lam[..., self.d + 1]
        with np.errstate(invalid="ignore", over="ignore"):
            u = self.u_s(Lam)
            ok = (LE < 0) & np.all(np.isfinite(u), axis=-1) & (u[..., 0] > 0)
        return ok

    # --- primitive helpers for initial / boundary data -------------------------------------
    def conserved(self, rho, vel, p):
        """(rho, v, p) -> (rho, rho v, p/(gamma-1) + rho |v|^2/2); vel has trailing dim d."""
        rho = np.asarray(rho, dtype=np.float64)
        vel = np.asarray(vel, dtype=np.float64)
        p = np.asarray(p, dtype=np.float64)
        out = np.empty(rho.shape + (self.m,))
        out[..., 0] = rho
        out[..., 1:1 + self.d] = rho[..., None] * vel
        out[..., self.d + 1] = p / (self.gamma - 1.0) + 0.5 * rho * np.sum(vel * vel, axis=-1)
        return out
