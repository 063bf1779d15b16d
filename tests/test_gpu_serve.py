"""Request loop (ibm_server_*): continuous batching of independent cases.

Each request must give the same result in the mix as alone: the cases share
nothing on the device and every kernel of the step is deterministic (no
floating-point atomics), so forces and time are compared bit for bit.  The
admission tests check the memory gate and the slot limit.
"""
import numpy as np
import pytest

from paper_1912_11908_gb300 import ibm
from paper_1912_11908_gb300 import workloads as W

pytestmark = pytest.mark.gpu

STEPS = 23


def _specs(n=10, max_cells=256 * 128):
    """A small slice of the seeded serving mix: stationary and oscillating, subsonic and supersonic."""
    reqs = [r["spec"] for r in W.serving_mix(96) if r["spec"]["nx"] * r["spec"]["ny"] <= max_cells]
    osc = [s for s in reqs if s["motion"] != W.MOTION_STATIC]
    sup = [s for s in reqs if s["mach"] > 1.0]
    picked = {s["name"] for s in osc[:3] + sup[:2]}
    rest = [s for s in reqs if s["name"] not in picked]
    out = osc[:3] + sup[:2] + rest[: n - len(picked)]
    assert len(out) == n and osc and sup
    return out


def _alone(spec, nsteps):
    c = ibm.Case(spec)
    try:
        c.classify()
        c.step(nsteps)
        return c.forces(), c.time()[0]
    finally:
        c.close()


def _drain(srv, specs_by_id=None, budget=None, cap=None):
    max_running = 0
    while True:
        na, npend = srv.progress()
        max_running = max(max_running, na)
        if budget is not None:
            running = [rid for rid in specs_by_id if srv.poll(rid)["state"] == ibm.REQ_RUNNING]
            assert sum(ibm.case_device_bytes(specs_by_id[r]) for r in running) <= budget
        if cap is not None:
            assert na <= cap
        if na == 0 and npend == 0:
            return max_running


def test_mix_results_identical_to_alone():
    specs = _specs()
    ref = [_alone(s, STEPS) for s in specs]
    srv = ibm.Server(max_active=4, steps_per_chunk=7)
    try:
        ids = [srv.submit(s, STEPS) for s in specs]
        max_running = _drain(srv, cap=4)
        assert max_running >= 2, "no two cases ran together"
        for rid, (f, t) in zip(ids, ref):
            r = srv.poll(rid)
            assert r["state"] == ibm.REQ_DONE and r["status"] == 0, r
            assert r["steps_done"] == STEPS
            np.testing.assert_array_equal(r["forces"], f)
            assert r["t"] == t
            assert r["submit_s"] <= r["start_s"] <= r["finish_s"]
    finally:
        srv.close()


def test_requests_arriving_while_others_run():
    """Requests submitted between passes of the loop join the running cases."""
    specs = _specs(8)
    ref = [_alone(s, STEPS) for s in specs]
    srv = ibm.Server(max_active=3, steps_per_chunk=5)
    try:
        ids = []
        overlapped = False
        for s in specs:
            ids.append(srv.submit(s, STEPS))
            na, _ = srv.progress()
            overlapped |= na >= 2
            srv.progress()
        _drain(srv, cap=3)
        assert overlapped
        for rid, (f, t) in zip(ids, ref):
            r = srv.poll(rid)
            assert r["state"] == ibm.REQ_DONE, r
            np.testing.assert_array_equal(r["forces"], f)
            assert r["t"] == t
    finally:
        srv.close()


def test_memory_gated_admission():
    specs = _specs(6)
    sizes = sorted(ibm.case_device_bytes(s) for s in specs)
    budget = sizes[-1] + sizes[-2]  # room for two of the largest, so never for all six at once
    srv = ibm.Server(device_bytes_budget=budget, max_active=64, steps_per_chunk=4)
    try:
        by_id = {srv.submit(s, 9): s for s in specs}
        _drain(srv, by_id, budget=budget)
        for rid in by_id:
            assert srv.poll(rid)["state"] == ibm.REQ_DONE
    finally:
        srv.close()


def test_request_larger_than_budget_is_refused():
    spec = _specs(6)[0]
    srv = ibm.Server(device_bytes_budget=ibm.case_device_bytes(spec) - 1, max_active=2, steps_per_chunk=4)
    try:
        with pytest.raises(ibm.IbmError) as e:
            srv.submit(spec, 5)
        assert e.value.status == ibm.IBM_ENOMEM
    finally:
        srv.close()


def test_zero_step_request_and_unknown_id():
    spec = _specs(6)[0]
    srv = ibm.Server(max_active=2, steps_per_chunk=4)
    try:
        rid = srv.submit(spec, 0)
        srv.drain()
        r = srv.poll(rid)
        assert r["state"] == ibm.REQ_DONE and r["steps_done"] == 0 and r["t"] == 0.0
        with pytest.raises(ibm.IbmError):
            srv.poll(rid + 1000)
    finally:
        srv.close()
