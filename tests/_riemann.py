"""Exact solution of the 1-D Euler Riemann problem (test infrastructure, independent of oracle/).

The star pressure p* solves f_L(p) + f_R(p) + (u_R - u_L) = 0, where f_K is the velocity change across the
wave on side K: a shock (p > p_K, from the Rankine-Hugoniot conditions) or a centred rarefaction
(p <= p_K, from the isentropic relation and the Riemann invariant u +- 2c/(gamma-1)); f is increasing in p,
so the root is bracketed and found by Brent's method. u* follows from either side. The self-similar
solution at x/t is then sampled wave by wave. This is the standard construction of the exact solver for
a polytropic gas (e.g. Toro, Riemann Solvers and Numerical Methods for Fluid Dynamics, Ch. 4), written
here from that derivation.
"""
import numpy as np
from scipy.optimize import brentq


class RiemannSolution:
    def __init__(self, left, right, gamma):
        """left / right: primitive states (rho, u, p)."""
        self.g = gamma
        self.L = tuple(float(v) for v in left)
        self.R = tuple(float(v) for v in right)
        g = gamma
        self.cL = np.sqrt(g * self.L[2] / self.L[0])
        self.cR = np.sqrt(g * self.R[2] / self.R[0])
        fp = lambda p: self._f(p, self.L, self.cL) + self._f(p, self.R, self.cR) + (self.R[1] - self.L[1])
        lo, hi = 1e-12, max(self.L[2], self.R[2])
        while fp(hi) < 0.0:
            hi *= 2.0
        self.ps = brentq(fp, lo, hi, xtol=1e-15, rtol=1e-15, maxiter=500)
        self.us = 0.5 * (self.L[1] + self.R[1]) + 0.5 * (self._f(self.ps, self.R, self.cR) - self._f(self.ps, self.L, self.cL))

    def _f(self, p, W, c):
        rho, _, pk = W
        g = self.g
        if p > pk:
            A = 2.0 / ((g + 1.0) * rho)
            B = (g - 1.0) / (g + 1.0) * pk
            return (p - pk) * np.sqrt(A / (p + B))
        return 2.0 * c / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)

    def star_density(self, side):
        W = self.L if side < 0 else self.R
        g, ratio = self.g, self.ps / W[2]
        if self.ps > W[2]:
            g6 = (g - 1.0) / (g + 1.0)
            return W[0] * (ratio + g6) / (g6 * ratio + 1.0)
        return W[0] * ratio ** (1.0 / g)

    def shock_speed(self, side):
        """Speed of the shock on the given side (only meaningful when p* exceeds that side's pressure)."""
        W, c = (self.L, self.cL) if side < 0 else (self.R, self.cR)
        g = self.g
        q = np.sqrt((g + 1.0) / (2.0 * g) * self.ps / W[2] + (g - 1.0) / (2.0 * g))
        return W[1] - c * q if side < 0 else W[1] + c * q

    def sample(self, s):
        """Primitive (rho, u, p) at similarity coordinates s = (x - x0) / t (array)."""
        s = np.asarray(s, dtype=np.float64)
        g = self.g
        rho, u, p = np.empty_like(s), np.empty_like(s), np.empty_like(s)
        for side in (-1, 1):
            W, c = (self.L, self.cL) if side < 0 else (self.R, self.cR)
            on = (s < self.us) if side < 0 else (s >= self.us)
            rs = self.star_density(side)
            if self.ps > W[2]:
                S = self.shock_speed(side)
                outer = on & ((s < S) if side < 0 else (s > S))
                inner = on & ~outer
                rho[outer], u[outer], p[outer] = W
                rho[inner], u[inner], p[inner] = rs, self.us, self.ps
            else:
                cs = c * (self.ps / W[2]) ** ((g - 1.0) / (2.0 * g))
                head = W[1] - c if side < 0 else W[1] + c
                tail = self.us - cs if side < 0 else self.us + cs
                outer = on & ((s < head) if side < 0 else (s > head))
                star = on & ((s > tail) if side < 0 else (s < tail))
                fan = on & ~outer & ~star
                rho[outer], u[outer], p[outer] = W
                rho[star], u[star], p[star] = rs, self.us, self.ps
                sf = s[fan]
                if side < 0:
                    uf = 2.0 / (g + 1.0) * (c + 0.5 * (g - 1.0) * W[1] + sf)
                    cf = 2.0 / (g + 1.0) * (c + 0.5 * (g - 1.0) * (W[1] - sf))
                else:
                    uf = 2.0 / (g + 1.0) * (-c + 0.5 * (g - 1.0) * W[1] + sf)
                    cf = 2.0 / (g + 1.0) * (c - 0.5 * (g - 1.0) * (W[1] - sf))
                rho[fan] = W[0] * (cf / c) ** (2.0 / (g - 1.0))
                u[fan] = uf
                p[fan] = W[2] * (cf / c) ** (2.0 * g / (g - 1.0))
        return rho, u, p


def sod_density_moments(nx, x_lo, x_hi, t, gamma, n12=6, n3=400, sub=16):
    """Expectation and variance of the cell averages of rho(x, t) for the uncertain Sod tube (rho_L = 1 + 0.1 xi_1, p_L = 1 + 0.1 xi_2,
    interface 0.5 + 0.05 xi_3, right state (0.125, 0, 0.1), xi ~ U[-1, 1]^3) by brute-force collocation of
    the exact solution: Gauss-Legendre in xi_1 and xi_2 (the solution is smooth in them away from the
    waves), a midpoint rule of n3 points in xi_3 (the waves shift with it), and sub midpoints per cell."""
    g1, w1 = np.polynomial.legendre.leggauss(n12)
    x3 = -1.0 + (np.arange(n3) + 0.5) * 2.0 / n3
    dx = (x_hi - x_lo) / nx
    xs = x_lo + (np.arange(nx)[:, None] + (np.arange(sub)[None, :] + 0.5) / sub) * dx       # (nx, sub)
    m1, m2 = np.zeros(nx), np.zeros(nx)
    for a, wa in zip(g1, w1):
        for b, wb in zip(g1, w1):
            sol = RiemannSolution((1.0 + 0.1 * a, 0.0, 1.0 + 0.1 * b), (0.125, 0.0, 0.1), gamma)
            x0 = 0.5 + 0.05 * x3                                                            # (n3,)
            rho, _, _ = sol.sample((xs[:, :, None] - x0[None, None, :]) / t)
            cell = rho.mean(axis=1)                                                         # (nx, n3) cell averages
            m1 += (wa / 2.0) * (wb / 2.0) * cell.mean(axis=1)
            m2 += (wa / 2.0) * (wb / 2.0) * (cell ** 2).mean(axis=1)
    return m1, m2 - m1 ** 2
