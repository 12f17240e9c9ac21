"""Parameters of the benchmark workloads (numbers only: no method arithmetic lives here).

Both the CUDA path (through ``ipm.make_problem``) and the CPU oracle (through the test helpers)
are set up from these dictionaries, so the two sides run the same problem. Primitive states are
(u) for Burgers and (rho, v, p) for Euler; every parameter is affine in xi ~ U[-1,1]^p:
``value + sum_d d_value[d] * xi_d``.
"""
import numpy as np

# 1-D Burgers, barrier entropy, 1 uncertain dim (shock position); Q = 10 Gauss nodes, N = 6.
BURGERS_1D = dict(
    name="burgers1d_ipm_fp64", kind="burgers1d", nx=200, x_lo=0.0, x_hi=3.0, bc=("outflow", "outflow"),
    cfl=0.5, t_end=0.11, gamma=1.4, p=1, M=5, nq=10, entropy="barrier", u_minus=0.5, u_plus=13.0,
    x0=0.5, dx0=(0.2, 0.0, 0.0), left=(12.0,), dleft=((0.0, 0.0, 0.0),), right=(1.0,), dright=((0.0, 0.0, 0.0),),
    newton_tol=1e-10,
)

# 1-D Euler Sod tube, 3 uncertain dims (rho_L, p_L, interface), total degree 5 (N = 56), 6^3 nodes.
SOD_1D = dict(
    name="sod1d_ipm", kind="euler1d", nx=2000, x_lo=0.0, x_hi=1.0, bc=("outflow", "outflow"),
    cfl=0.5, t_end=0.14, gamma=1.4, p=3, M=5, nq=6, entropy="euler", u_minus=0.0, u_plus=0.0,
    x0=0.5, dx0=(0.0, 0.0, 0.05),
    left=(1.0, 0.0, 1.0), dleft=((0.1, 0.0, 0.0), (0.0, 0.0, 0.0), (0.0, 0.1, 0.0)),
    right=(0.125, 0.0, 0.1), dright=((0.0, 0.0, 0.0),) * 3,
    newton_tol=1e-10,
)


# 2-D steady Euler over a 15-degree ramp (One-Shot IPM): inflow Mach 2 + 0.1 xi_1 at 10 + 1 xi_2 degrees,
# rho = p = 1; 256 x 128 cells on x in [0, 2] under y = 1 (ramp from x = 0.5); total degree 4 in 2 dims
# (N = 15 moments x 4 variables), 5 x 5 Gauss nodes; sides: inflow (Dirichlet), outflow, slip wall,
# far field (Dirichlet); pseudo-time steps until the steady residual falls below 1e-8.
RAMP_2D = dict(
    name="ramp2d_oneshot", kind="euler2d", nx=256, ny=128, x_lo=0.0, x_hi=2.0, y_lo=0.0, y_hi=1.0, mesh="ramp",
    ramp_x0=0.5, ramp_deg=15.0, sides=("dirichlet", "outflow", "slip", "dirichlet"), cfl=0.4, t_end=0.0, gamma=1.4,
    p=2, M=4, nq=5, entropy="euler", ic="freestream", param=(1.0, 1.0, 2.0, 10.0),
    dparam=((0.0, 0.0, 0.0), (0.0, 0.0, 0.0), (0.1, 0.0, 0.0), (0.0, 1.0, 0.0)), newton_tol=1e-10,
    residual_tol=1e-8,
)

# 2-D Kelvin-Helmholtz-type shear layer on the periodic unit square, 512 x 512 cells: rho = 2, v_1 = -0.5
# inside |y - 0.5| < 0.25 + 0.02 xi_3, rho = 1, v_1 = 0.5 outside, p = 2.5, v_2 = 0.01 (1 + 0.5 xi_1)
# sin(4 pi (x + 0.1 xi_2)); 3 dims, 7^3 = 343 Gauss nodes, total degree M (2..6).
KH_2D = dict(
    name="kh2d", kind="euler2d", nx=512, ny=512, x_lo=0.0, x_hi=1.0, y_lo=0.0, y_hi=1.0, mesh="cartesian",
    ramp_x0=0.0, ramp_deg=0.0, sides=("periodic",) * 4, cfl=0.4, t_end=0.0, gamma=1.4, p=3, M=2, nq=7,
    entropy="euler", ic="shear", left=(2.0, -0.5, 0.0, 2.5), right=(1.0, 0.5, 0.0, 2.5),
    param=(0.01, 0.0, 0.25, 4.0 * np.pi), dparam=((0.005, 0.0, 0.0), (0.0, 0.1, 0.0), (0.0, 0.0, 0.02), (0.0, 0.0, 0.0)),
    newton_tol=1e-10, steps=200,
)

# 2-D data varying in x only (a Sod-type jump at x = 0.5, rho_L = 1 + 0.1 xi_1, p_L = 1 + 0.1 xi_2), periodic in y
XRIEMANN_2D = dict(
    name="xriemann2d", kind="euler2d", nx=30, ny=2, x_lo=0.0, x_hi=1.0, y_lo=0.0, y_hi=0.2, mesh="cartesian",
    ramp_x0=0.0, ramp_deg=0.0, sides=("outflow", "outflow", "periodic", "periodic"), cfl=0.4, t_end=0.0,
    gamma=1.4, p=2, M=2, nq=3, entropy="euler", ic="riemann", x0=0.5, left=(1.0, 0.0, 0.0, 1.0),
    dleft=((0.1, 0.0, 0.0), (0.0, 0.0, 0.0), (0.0, 0.0, 0.0), (0.0, 0.1, 0.0)), right=(0.125, 0.0, 0.0, 0.1),
    dright=((0.0, 0.0, 0.0),) * 4, param=(0.0, 0.0, 0.0, 0.0), dparam=None, newton_tol=1e-10,
)

# The Sod tube of SOD_1D under the literal reading of "56 moments x 4": the four-variable 2-D Euler system
# (rho, rho v_1, rho v_2, E) with v_2 = 0 on a 2000 x 1 Cartesian mesh (square cells, periodic in y, outflow
# in x), the same uncertain data (rho_L, p_L, interface), total degree 5 in 3 dims (N = 56 x 4 variables),
# 6^3 Gauss nodes, local Lax-Friedrichs faces, CFL 0.5, to t_end = 0.14.
SOD_1D_AS_2D = dict(
    name="sod1d_as_2d", kind="euler2d", nx=2000, ny=1, x_lo=0.0, x_hi=1.0, y_lo=0.0, y_hi=1.0 / 2000,
    mesh="cartesian", ramp_x0=0.0, ramp_deg=0.0, sides=("outflow", "outflow", "periodic", "periodic"), cfl=0.5,
    t_end=0.14, gamma=1.4, p=3, M=5, nq=6, entropy="euler", ic="riemann", x0=0.5, dx0=(0.0, 0.0, 0.05),
    left=(1.0, 0.0, 0.0, 1.0), dleft=((0.1, 0.0, 0.0), (0.0, 0.0, 0.0), (0.0, 0.0, 0.0), (0.0, 0.1, 0.0)),
    right=(0.125, 0.0, 0.0, 0.1), dright=((0.0, 0.0, 0.0),) * 4, param=(0.0, 0.0, 0.0, 0.0), dparam=None,
    newton_tol=1e-10,
)


def variant(base: dict, **changes) -> dict:
    """Copy of a workload with some parameters changed (smaller meshes for parity cases)."""
    out = dict(base)
    out.update(changes)
    return out


def random_dual_perturbation(shape, seed: int, scale: float) -> np.ndarray:
    """Seeded Gaussian perturbation used to build manufactured dual states for round-trip tests."""
    return scale * np.random.default_rng(seed).standard_normal(shape)


def serving_requests(n: int, seed: int = 1234, rate_hz: float = 0.0, steps: int = 10,
                     max_cells: int = 4000, max_degree: int = 6) -> list:
    """A seeded stream of IPM requests shaped like the serving workload: each request is a 1-D Burgers
    or 1-D Euler (Sod-family) problem with cells uniform in [200, max_cells], total degree uniform in
    2..max_degree, 1..3 uniform uncertain dimensions and a tensor Gauss rule of (degree + 1) nodes per
    dimension, running `steps` time steps. Arrivals are a Poisson process of rate rate_hz (all at t = 0
    when rate_hz is 0). Returns [(arrival_s, workload dict)].

    Uncertain parameters (affine in xi_d ~ U[-1, 1]): Burgers -- jump position 0.5 + 0.2 xi_1 on
    [0, 3], left state 12 + 0.5 xi_2, right state 1 + 0.5 xi_3 (inside the barrier bounds 0.5, 13);
    Euler -- the first p of (rho_L = 1 + 0.1 xi, p_L = 1 + 0.1 xi, interface 0.5 + 0.05 xi)."""
    rng = np.random.default_rng(seed)
    out, t = [], 0.0
    for k in range(n):
        if rate_hz > 0.0:
            t += float(rng.exponential(1.0 / rate_hz))
        fam = "burgers1d" if rng.random() < 0.5 else "euler1d"
        nx = int(rng.integers(200, max_cells + 1))
        deg = int(rng.integers(2, max_degree + 1))
        p = int(rng.integers(1, 4))
        if fam == "burgers1d":
            d = [0.0, 0.0, 0.0]
            d[0] = 0.2
            dl = [0.0, 0.5 if p >= 2 else 0.0, 0.0]
            dr = [0.0, 0.0, 0.5 if p >= 3 else 0.0]
            w = variant(BURGERS_1D, name=f"req{k}_burgers", nx=nx, p=p, M=deg, nq=deg + 1, t_end=0.0,
                        dx0=tuple(d), dleft=(tuple(dl),), dright=(tuple(dr),))
        else:
            dl = [[0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]]
            dx0 = [0.0, 0.0, 0.0]
            dl[0][0] = 0.1                       # rho_L on xi_1
            if p >= 2:
                dl[2][1] = 0.1                   # p_L on xi_2
            if p >= 3:
                dx0[2] = 0.05                    # interface on xi_3
            w = variant(SOD_1D, name=f"req{k}_euler", nx=nx, p=p, M=deg, nq=deg + 1, t_end=0.0,
                        dx0=tuple(dx0), dleft=tuple(tuple(r) for r in dl))
        w["steps"] = steps
        out.append((t, w))
    return out


# ------------------------------------------------------------------------------------------------
# Library objects for a workload dictionary (the CUDA path only; these import nothing but the binding).

def problem(w: dict):
    """The ipm_problem of a workload dictionary (1-D or 2-D)."""
    from . import ipm
    if w["kind"] == "euler2d":
        return ipm.make_problem_2d(w["nx"], w["ny"], w["x_lo"], w["x_hi"], w["y_lo"], w["y_hi"], sides=w["sides"],
                                   mesh=w["mesh"], ramp_x0=w["ramp_x0"], ramp_deg=w["ramp_deg"], cfl=w["cfl"],
                                   t_end=w["t_end"], gamma=w["gamma"], ic=w["ic"], param=w["param"],
                                   dparam=w.get("dparam"), x0=w.get("x0", 0.5), left=w.get("left", (0, 0, 0, 0)),
                                   dleft=w.get("dleft"), right=w.get("right", (0, 0, 0, 0)), dright=w.get("dright"),
                                   dx0=w.get("dx0", (0.0, 0.0, 0.0)))
    return ipm.make_problem(w["kind"], w["nx"], w["x_lo"], w["x_hi"], bc=w["bc"], cfl=w["cfl"], t_end=w["t_end"],
                            gamma=w["gamma"], x0=w["x0"], dx0=w["dx0"], left=w["left"], dleft=w.get("dleft"),
                            right=w["right"], dright=w.get("dright"))


def quadrature(w: dict):
    """The workload's rule: tensor Gauss with nq nodes per dimension, or nested Clenshaw-Curtis rules
    when the workload names cc_levels."""
    from . import ipm
    return ipm.quadrature(w["nq"], cc_levels=w.get("cc_levels"))


def context(w: dict, precision: str = "fp64", tau=None, **opt):
    """An ipm.Context holding the workload's initial state on the current device."""
    from . import ipm
    o = ipm.default_options(precision, newton_tol=tau if tau is not None else w.get("newton_tol", 1e-10), **opt)
    if w["kind"] == "euler2d":
        return ipm.Context(problem(w), w["p"], w["M"], quadrature(w), w["entropy"], 0.0, 0.0, o)
    return ipm.Context(problem(w), w["p"], w["M"], quadrature(w), w["entropy"], w.get("u_minus", 0.0),
                       w.get("u_plus", 0.0), o)


def collocation(w: dict, steady_tol: float = 0.0):
    """Stochastic Collocation of a workload on the GPU (ipm_sc_*), on the workload's quadrature."""
    from . import ipm
    return ipm.Collocation(problem(w), w["p"], w["M"], quadrature(w), steady_tol)


def request(w: dict, precision: str = "mixed", max_steps=None):
    """An ipm_request for the serving API (1-D workloads); max_steps defaults to w["steps"] when present."""
    from . import ipm
    o = ipm.default_options(precision, newton_tol=w.get("newton_tol", 1e-10))
    steps = max_steps if max_steps is not None else w.get("steps", 2 ** 62)
    return ipm.make_request(problem(w), w["p"], w["M"], w["nq"], w["entropy"], w.get("u_minus", 0.0),
                            w.get("u_plus", 0.0), o, max_steps=steps)
