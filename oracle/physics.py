"""Physical fluxes, wave speeds and deterministic numerical fluxes (test infrastructure).

* Burgers: f(u) = u^2/2 (App. A).
* Euler: conserved (rho, rho v, rho e), p = (gamma-1)(rho e - rho|v|^2/2) (Sec. 7.1); the flux in
  direction n is (rho v.n, rho v (v.n) + p n, (rho e + p) v.n); the largest wave speed is |v.n| + c,
  c = sqrt(gamma p / rho).
* Lax-Friedrichs flux g(u_l, u_r) = (f(u_l) + f(u_r))/2 - dx/(2 dt) (u_r - u_l) (App. A, per-node
  form of Eq. numFluxAnalytic), used node by node inside the kinetic flux (Eq. numericalFluxIPM).
* On 2-D meshes (no single dx) the viscosity is local: a = max(|v.n|+c) of the two states
  (Rusanov); g = (F(u_l).n + F(u_r).n)/2 - a/2 (u_r - u_l).

Pinned by: tests/test_oracle_scheme.py (consistency g(u,u) = f(u), constant states preserved,
deterministic limit) and the SG / Rankine-Hugoniot pins.
"""
import numpy as np


class Burgers1D:
    m = 1
    dim = 1

    def flux(self, u):
        return 0.5 * u * u

    def speed(self, u):
        return np.abs(u[..., 0])


class Euler:
    def __init__(self, gamma: float, dim: int):
        self.gamma = float(gamma)
        self.dim = dim
        self.m = dim + 2

    def pressure(self, u):
        rho = u[..., 0]
        mom = u[..., 1:1 + self.dim]
        E = u[..., self.dim + 1]
        return (self.gamma - 1.0) * (E - 0.5 * np.sum(mom * mom, axis=-1) / rho)

    def normal_flux(self, u, n):
        """F(u) . n for a unit normal n of length dim (broadcast over leading dims)."""
        n = np.asarray(n, dtype=np.float64)
        rho = u[..., 0]
        mom = u[..., 1:1 + self.dim]
        E = u[..., self.dim + 1]
        p = self.pressure(u)
        vn = np.sum(mom * n, axis=-1) / rho
        out = np.empty(u.shape)
        out[..., 0] = rho * vn
        out[..., 1:1 + self.dim] = mom * vn[..., None] + p[..., None] * n
        out[..., self.dim + 1] = (E + p) * vn
        return out

    def flux(self, u):
        """1-D flux (dim must be 1)."""
        assert self.dim == 1
        return self.normal_flux(u, np.array([1.0]))

    def normal_speed(self, u, n):
        n = np.asarray(n, dtype=np.float64)
        rho = u[..., 0]
        vn = np.sum(u[..., 1:1 + self.dim] * n, axis=-1) / rho
        c = np.sqrt(self.gamma * self.pressure(u) / rho)
        return np.abs(vn) + c

    def speed(self, u):
        """Largest characteristic speed over the coordinate directions."""
        rho = u[..., 0]
        c = np.sqrt(self.gamma * self.pressure(u) / rho)
        vmax = np.max(np.abs(u[..., 1:1 + self.dim]), axis=-1) / rho
        return vmax + c


def lax_friedrichs(phys, ul, ur, dx, dt):
    """Global Lax-Friedrichs flux, node by node (App. A)."""
    return 0.5 * (phys.flux(ul) + phys.flux(ur)) - (dx / (2.0 * dt)) * (ur - ul)


def rusanov(phys, ul, ur, n):
    """Local Lax-Friedrichs flux across a face with unit normal n (2-D meshes)."""
    a = np.maximum(phys.normal_speed(ul, n), phys.normal_speed(ur, n))
    return 0.5 * (phys.normal_flux(ul, n) + phys.normal_flux(ur, n)) - 0.5 * a[..., None] * (ur - ul)
