"""Test helpers: set up the same workload on the CPU oracle and on the CUDA library.

The oracle side is built from the workload numbers alone; the library side through the C ABI.
No value flows from the CUDA path into the oracle."""
import numpy as np

from oracle import basis, dual, entropy, physics
from oracle import scheme1d as s1
# the CUDA side of a workload: the library's own helpers (they import nothing from oracle/)
from paper_1912_09238_gb300.workloads import collocation as gpu_collocation  # noqa: F401
from paper_1912_09238_gb300.workloads import context as gpu_context  # noqa: F401
from paper_1912_09238_gb300.workloads import problem as gpu_problem  # noqa: F401
from paper_1912_09238_gb300.workloads import quadrature as gpu_quadrature  # noqa: F401


def _affine(vals, dvals, nvar):
    vals = np.asarray(vals, dtype=np.float64)
    d = np.zeros((nvar, 3))
    if dvals is not None:
        for v in range(min(nvar, len(dvals))):
            d[v, :len(dvals[v])] = dvals[v]
    return lambda xi: vals[None, :nvar] + xi @ d[:nvar, :xi.shape[1]].T


def oracle_problem(w, tau=None):
    """oracle.scheme1d.Problem1D for a workload dictionary (see paper_1912_09238_gb300.workloads)."""
    sp = basis.StochasticSpace(w["p"], w["M"], w["nq"])
    if w["kind"] == "burgers1d":
        phys = physics.Burgers1D()
        ent = entropy.BoundedBarrier(w["u_minus"], w["u_plus"]) if w["entropy"] == "barrier" else entropy.Quadratic(1)
        L = _affine(w["left"], w.get("dleft"), 1)
        R = _affine(w["right"], w.get("dright"), 1)
        left, right = L, R
    else:
        phys = physics.Euler(w["gamma"], 1)
        ent = entropy.Euler(w["gamma"], 1) if w["entropy"] == "euler" else entropy.Quadratic(3)
        E = entropy.Euler(w["gamma"], 1)
        L = _affine(w["left"], w.get("dleft"), 3)
        R = _affine(w["right"], w.get("dright"), 3)
        left = lambda xi: E.conserved(L(xi)[:, 0], L(xi)[:, 1:2], L(xi)[:, 2])
        right = lambda xi: E.conserved(R(xi)[:, 0], R(xi)[:, 1:2], R(xi)[:, 2])
    dx0 = np.asarray(w["dx0"], dtype=np.float64)
    x0 = lambda xi: w["x0"] + xi @ dx0[:xi.shape[1]]
    prob = s1.Problem1D(phys=phys, ent=ent, space=sp, nx=w["nx"], x_lo=w["x_lo"], x_hi=w["x_hi"],
                        ic=s1.RiemannIC(left, right, x0), bc="/".join(w["bc"]), cfl=w["cfl"], t_end=w["t_end"])
    prob.newton = dual.NewtonOptions(tau=tau if tau is not None else w.get("newton_tol", 1e-10))
    return prob


def oracle_problem_2d(w, tau=None):
    """oracle.scheme2d.Problem2D for a 2-D workload dictionary (a nested Clenshaw-Curtis space of the
    finest level when the workload names cc_levels)."""
    from oracle import scheme2d as s2
    if w.get("cc_levels"):
        sp = basis.NestedCCSpace(w["p"], w["M"], max(w["cc_levels"]))
    else:
        sp = basis.StochasticSpace(w["p"], w["M"], w["nq"])
    phys = physics.Euler(w["gamma"], 2)
    ent = entropy.Euler(w["gamma"], 2) if w["entropy"] == "euler" else entropy.Quadratic(4)
    if w["mesh"] == "ramp":
        mesh = s2.ramp_mesh(w["nx"], w["ny"], w["x_lo"], w["x_hi"], w["y_hi"], w["ramp_x0"], w["ramp_deg"])
    else:
        mesh = s2.cartesian_mesh(w["nx"], w["ny"], w["x_lo"], w["x_hi"], w["y_lo"], w["y_hi"])
    dp = w.get("dparam") or ((0.0, 0.0, 0.0),) * 4
    if w["ic"] == "freestream":
        ic = s2.FreestreamIC(rho=w["param"][0], p=w["param"][1], mach=w["param"][2], angle_deg=w["param"][3],
                             dmach=dp[2], dangle=dp[3])
    elif w["ic"] == "shear":
        L, R = w["left"], w["right"]
        ic = s2.ShearIC(rho_in=L[0], v_in=L[1], rho_out=R[0], v_out=R[1], p=L[3], amp=w["param"][0],
                        phase=w["param"][1], half_width=w["param"][2], k=w["param"][3],
                        y_mid=0.5 * (w["y_lo"] + w["y_hi"]), damp=dp[0], dphase=dp[1], dhalf_width=dp[2])
    else:
        ic = s2.RiemannXIC(left=tuple(w["left"]), right=tuple(w["right"]), x0=w["x0"],
                           dleft=w.get("dleft") or ((0.0, 0.0, 0.0),) * 4, dright=w.get("dright") or ((0.0, 0.0, 0.0),) * 4,
                           dx0=tuple(w.get("dx0", (0.0, 0.0, 0.0))))
    return s2.Problem2D(phys=phys, ent=ent, space=sp, mesh=mesh, ic=ic, sides=tuple(w["sides"]), cfl=w["cfl"],
                        t_end=w["t_end"], newton=dual.NewtonOptions(tau=tau if tau is not None else w.get("newton_tol", 1e-10)))


def rel_err(a, b):
    """Normwise relative difference max|a - b| / max|b| (b is the oracle)."""
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
