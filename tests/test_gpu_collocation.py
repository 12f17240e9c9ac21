"""GPU parity of Stochastic Collocation (ipm_sc_*) against the oracle (oracle/collocation.py), through
the C ABI: nodal states of every node (ghosts included) and the SC moments at 1e-10 relative, and the
step count of every node exactly (each node runs on its own time steps)."""
import numpy as np
import pytest

from oracle import collocation as sc
from paper_1912_09238_gb300 import workloads
from tests._cases import gpu_collocation, oracle_problem, oracle_problem_2d, rel_err

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_09238_gb300 import build
    build.build()


def _compare_1d(w, steady_tol=0.0, max_steps=2 ** 62):
    prob = oracle_problem(w)
    ref = sc.run_1d(prob, steady_tol=steady_tol, max_steps=max_steps)
    g = gpu_collocation(w, steady_tol)
    s = g.run(max_steps)
    steps, t, _ = g.node_info()
    assert np.array_equal(steps, ref.steps)
    assert rel_err(t, ref.t) < 1e-13
    assert rel_err(g.get_nodal(), ref.U) < TOL
    assert rel_err(g.get_moments(), ref.moments(prob.space)) < TOL
    assert s.max_node_steps == ref.steps.max() and s.active_nodes == 0
    g.close()
    return ref


def test_burgers_workload():
    ref = _compare_1d(workloads.BURGERS_1D)
    assert np.all(ref.t == workloads.BURGERS_1D["t_end"])


def test_sod_small_three_dims():
    w = workloads.variant(workloads.SOD_1D, nx=64, M=2, nq=3, t_end=0.1)
    ref = _compare_1d(w)
    assert len(set(ref.steps.tolist())) > 1              # the nodes take different numbers of steps


def test_periodic_and_dirichlet_ends():
    _compare_1d(workloads.variant(workloads.BURGERS_1D, nx=80, bc=("periodic", "periodic"), x0=1.5, t_end=0.05))
    _compare_1d(workloads.variant(workloads.BURGERS_1D, nx=80, bc=("dirichlet", "outflow"), t_end=0.05))


def test_max_steps_stops_every_node():
    w = workloads.variant(workloads.BURGERS_1D, nx=50)
    prob = oracle_problem(w)
    ref = sc.run_1d(prob, max_steps=21)
    g = gpu_collocation(w)
    s = g.run(21)
    assert s.steps == 21 and s.active_nodes == prob.space.Q
    assert rel_err(g.get_nodal(), ref.U) < TOL
    s = g.step()
    assert s.steps == 22
    g.close()


def test_ramp_steady_nodes():
    w = workloads.variant(workloads.RAMP_2D, nx=12, ny=6, M=2, nq=3)
    prob = oracle_problem_2d(w)
    ref = sc.run_2d(prob, steady_tol=1e-6, max_steps=4000)
    g = gpu_collocation(w, 1e-6)
    s = g.run(4000)
    steps, _, res = g.node_info()
    assert np.array_equal(steps, ref.steps) and np.all(res < 1e-6)
    Q = prob.space.Q
    assert rel_err(g.get_nodal().reshape(ref.U.shape[:2] + (Q, 4)), ref.U) < TOL
    assert s.active_nodes == 0
    g.close()


def test_shear_layer_periodic_unsteady():
    w = workloads.variant(workloads.KH_2D, nx=10, ny=10, M=2, nq=2, t_end=0.1)
    prob = oracle_problem_2d(w)
    ref = sc.run_2d(prob)
    g = gpu_collocation(w)
    g.run()
    steps, t, _ = g.node_info()
    assert np.array_equal(steps, ref.steps) and np.all(t == 0.1)
    Q = prob.space.Q
    assert rel_err(g.get_nodal().reshape(ref.U.shape[:2] + (Q, 4)), ref.U) < TOL
    assert rel_err(g.get_moments().reshape(ref.U.shape[:2] + (-1, 4)), ref.moments(prob.space)) < TOL
    g.close()


def test_sod_full_size_sampled_nodes():
    """The 2000-cell Sod workload with 216 nodes: the GPU runs all of them; the oracle runs a sample of
    nodes (every node is independent), which must match column by column."""
    w = workloads.SOD_1D
    prob = oracle_problem(w)
    g = gpu_collocation(w)
    g.run()
    steps, t, _ = g.node_info()
    sample = [0, 1, 37, 108, 180, 215]
    ref = sc.run_1d(prob, nodes=sample)
    assert np.array_equal(steps[sample], ref.steps) and np.all(t == w["t_end"])
    got = g.get_nodal()[:, sample]
    assert rel_err(got, ref.U) < TOL
    g.close()
