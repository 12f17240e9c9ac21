"""Host-side checks of bench.py (no GPU): the timed GPU arm never loads the oracle, and the host-core
oracle baseline (cells split over processes) reproduces the oracle's own Algorithm-1 step."""
import ast
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
# the only functions of bench.py that may touch oracle/ or tests/: the host baseline, run in a subprocess
ORACLE_SIDE = {"oracle_sample", "_oracle_dual_chunk", "_oracle_chunk_problem", "_oracle_warm"}


def test_only_the_host_baseline_imports_the_oracle():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    for fn in [n for n in ast.walk(tree) if isinstance(n, ast.FunctionDef)]:
        for node in ast.walk(fn):
            mods = []
            if isinstance(node, ast.Import):
                mods = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                mods = [node.module or ""]
            for m in mods:
                if m.split(".")[0] in ("oracle", "tests"):
                    assert fn.name in ORACLE_SIDE, (fn.name, m)
    for node in tree.body:                      # nothing at module level either
        if isinstance(node, (ast.Import, ast.ImportFrom)):
            mods = [a.name for a in node.names] if isinstance(node, ast.Import) else [node.module or ""]
            assert all(m.split(".")[0] not in ("oracle", "tests") for m in mods), mods


def test_gpu_arm_imports_leave_the_oracle_unloaded():
    code = ("import sys; sys.path.insert(0, %r); import bench, __graft_entry__; "
            "from paper_1912_09238_gb300 import ipm, workloads, build; "
            "bad = [m for m in sys.modules if m == 'oracle' or m.startswith('oracle.') or m.startswith('tests')]; "
            "assert not bad, bad; print('ok')" % ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT, timeout=300)
    assert r.returncode == 0 and "ok" in r.stdout, r.stderr[-2000:]


def test_host_core_baseline_step_equals_the_oracle_step():
    """The baseline's step (dual solves of cell ranges in worker processes, the rest of Algorithm 1 in the
    parent) gives the oracle's own ipm_step result on a reduced Sod tube, to rounding."""
    sys.path.insert(0, ROOT)
    import bench
    from oracle import scheme1d as s1
    from paper_1912_09238_gb300 import workloads
    from tests._cases import oracle_problem
    w = workloads.variant(workloads.SOD_1D, nx=24, M=2, nq=3)
    orig = bench.workload
    bench.workload = lambda: w
    try:
        res = bench.oracle_sample(2, 2, keep_state=True)
    finally:
        bench.workload = orig
    prob = oracle_problem(w)
    st = s1.initial_state(prob)
    for _ in range(2):
        st = s1.ipm_step(prob, st)
    assert len(res["seconds"]) == 2 and res["procs"] == 2
    # numpy's batched kernels round differently on a range of cells than on all of them
    assert np.abs(res["uhat"] - st.uhat).max() <= 1e-10 * np.abs(st.uhat).max()
