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


def variant(base: dict, **changes) -> dict:
    """Copy of a workload with some parameters changed (smaller meshes for parity cases)."""
    out = dict(base)
    out.update(changes)
    return out


def random_dual_perturbation(shape, seed: int, scale: float) -> np.ndarray:
    """Seeded Gaussian perturbation used to build manufactured dual states for round-trip tests."""
    return scale * np.random.default_rng(seed).standard_normal(shape)
