"""The continuous-batching server (ipm_server_create / ipm_submit / ipm_poll) through the C ABI.

Checks: every request's final moments are identical whether it runs alone (its own context, the
same number of steps) or in a mix served concurrently; admission respects the memory cap and the
slot count; requests of the mix overlap in time; a served request matches the oracle; bad requests
are refused at submission."""
import numpy as np
import pytest

from oracle import scheme1d as s1
from paper_1912_09238_gb300 import workloads
from tests._cases import gpu_context, oracle_problem, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_09238_gb300 import build
    build.build()


def _request(w, precision):
    from paper_1912_09238_gb300 import ipm
    pr = ipm.make_problem(w["kind"], w["nx"], w["x_lo"], w["x_hi"], bc=w["bc"], cfl=w["cfl"], t_end=w["t_end"],
                          gamma=w["gamma"], x0=w["x0"], dx0=w["dx0"], left=w["left"], dleft=w.get("dleft"),
                          right=w["right"], dright=w.get("dright"))
    o = ipm.default_options(precision, newton_tol=w.get("newton_tol", 1e-10))
    return ipm.make_request(pr, w["p"], w["M"], w["nq"], w["entropy"], w.get("u_minus", 0.0), w.get("u_plus", 0.0),
                            o, max_steps=w["steps"])


def _alone(w, precision):
    ctx = gpu_context(w, precision=precision)
    for _ in range(w["steps"]):
        s = ctx.step()
        assert s.failed_cells == 0
    out = ctx.get_moments()
    ctx.close()
    return out


def _mix(n, seed, steps):
    return [w for _, w in workloads.serving_requests(n, seed=seed, steps=steps, max_cells=900, max_degree=4)]


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_results_same_alone_and_in_the_mix(precision):
    from paper_1912_09238_gb300 import ipm
    mix = _mix(10, 7, 6)
    srv = ipm.Server(mem_cap_bytes=0, max_active=6)
    tickets = [srv.submit(_request(w, precision)) for w in mix]
    srv.drain(600.0)
    results = [srv.poll(t) for t in tickets]
    srv.close()
    for w, (res, mom) in zip(mix, results):
        assert res.status == 0, (w["name"], res.status, res.error)
        assert res.stats.steps == w["steps"]
        ref = _alone(w, precision)
        # the same kernels on the same data: bit-identical, far inside the parity tolerance
        assert np.array_equal(mom, ref), (w["name"], rel_err(mom, ref))


def test_admission_by_memory_and_slots_and_overlap():
    from paper_1912_09238_gb300 import ipm
    mix = _mix(12, 11, 8)
    reqs = [_request(w, "mixed") for w in mix]
    fps = [ipm.footprint(r) for r in reqs]
    cap = int(2.5 * max(fps))                      # at most a few requests resident at once
    srv = ipm.Server(mem_cap_bytes=cap, max_active=3)
    tickets = [srv.submit(r) for r in reqs]
    srv.drain(600.0)
    res = [srv.poll(t)[0] for t in tickets]
    srv.close()
    assert all(r.status == 0 for r in res)
    # at every admission instant, the requests resident together fit the cap and the slots
    for r in res:
        t = r.start_s
        live = [q for q in res if q.start_s <= t < q.finish_s]
        assert sum(q.footprint_bytes for q in live) <= cap
        assert len(live) <= 3
    # FIFO admission
    starts = [r.start_s for r in res]
    assert starts == sorted(starts)
    # work of different requests overlapped in time
    overlaps = sum(1 for a in res for b in res if a is not b and a.start_s < b.finish_s and b.start_s < a.finish_s)
    assert overlaps > 0
    # latency bookkeeping is consistent
    assert all(r.submit_s <= r.start_s <= r.finish_s for r in res)


def test_served_request_matches_oracle():
    from paper_1912_09238_gb300 import ipm
    w = workloads.variant(workloads.SOD_1D, nx=48, M=3, nq=4, t_end=0.0)
    w["steps"] = 5
    prob = oracle_problem(w)
    st = s1.initial_state(prob)
    for _ in range(w["steps"]):
        st = s1.ipm_step(prob, st)
    srv = ipm.Server(max_active=2)
    t = srv.submit(_request(w, "mixed"))
    srv.drain(300.0)
    res, mom = srv.poll(t)
    srv.close()
    assert res.status == 0
    assert rel_err(mom, st.uhat) < 1e-6


def test_bad_requests_are_refused():
    from paper_1912_09238_gb300 import ipm
    w = workloads.variant(workloads.BURGERS_1D, nx=50)
    w["steps"] = 2
    srv = ipm.Server(mem_cap_bytes=1 << 20, max_active=2)
    r = _request(w, "mixed")
    r.basis.p = 5                                  # unsupported number of dimensions
    with pytest.raises(ipm.IpmError) as e:
        srv.submit(r)
    assert e.value.status == 1
    big = _request(workloads.variant(workloads.SOD_1D, nx=4000, steps=2), "mixed")
    with pytest.raises(ipm.IpmError) as e:
        srv.submit(big)                            # footprint above the 1 MiB cap
    assert e.value.status == 2
    srv.close()
