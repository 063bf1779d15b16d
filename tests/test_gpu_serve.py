"""Request loop (ibm_server_*): continuous batching of independent cases -- explicit requests with any motion
(a body under the fluid force included) and dual-time requests, each kind in block-table groups.

Each request must give the same result in the mix as alone.  Cases share
nothing on the device and every kernel of the step is deterministic (no
floating-point atomics), so with one stream per case -- the same kernels as a
case stepped alone -- forces and time are compared bit for bit, and so are
dual-time requests in batched groups (a dual-time case alone runs the same
block-table kernel with a table of one).  Batched explicit groups run the same
per-tile source in a separately compiled block-table kernel, whose FP32
roundings (fused multiply-adds) may differ by an ulp per operation; over the <= 23 steps of these tests that moves time by ~1e-8
relative and forces by at most ~1e-6 of the largest force component (the
largest measured, 1.1e-6, is on the lift of a body symmetric about the
stream, whose exact value is zero: rounding noise that the flow amplifies).
The tolerance is 1e-5 of the largest component.  Batched groups are also
checked against the FP64 oracle with the FP32-bulk bar (drag and lift within
1e-3).  The admission tests check the memory gate and the slot limit.
"""
import math

import numpy as np
import pytest

from paper_1912_11908_gb300 import ibm
from paper_1912_11908_gb300 import workloads as W

pytestmark = pytest.mark.gpu

STEPS = 23
RTOL_BATCHED = 1e-5


def _same(r, f, t, mode, spec):
    if mode & ibm.SERVE_BATCHED and spec["time_scheme"] != W.TIME_DUAL:
        np.testing.assert_allclose(r["forces"], f, rtol=RTOL_BATCHED, atol=RTOL_BATCHED * np.abs(f).max())
        assert abs(r["t"] - t) <= RTOL_BATCHED * abs(t)
    else:
        np.testing.assert_array_equal(r["forces"], f)
        assert r["t"] == t


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


def _coupled(nx=128, ny=64, mach=0.4, name="coupled"):
    """A cylinder free to translate in a uniform stream (Eq. 10), mass twice that of the gas it displaces."""
    return W.case_spec(W.cylinder(256), nx, ny, (-8.0, 24.0, -8.0, 8.0), mach, 200.0, W.FAR,
                       motion=W.MOTION_COUPLED, mass=2.0 * math.pi * 0.25, precision=W.PREC_FP32_BULK, name=name)


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


MODES = [ibm.SERVE_BATCHED | ibm.SERVE_AUTOTUNE, ibm.SERVE_BATCHED, 0]


@pytest.mark.parametrize("mode", MODES)
def test_mix_results_identical_to_alone(mode):
    specs = _specs(9) + [_coupled()]
    assert any(s["time_scheme"] == W.TIME_DUAL for s in specs)
    ref = [_alone(s, STEPS) for s in specs]
    srv = ibm.Server(max_active=4, steps_per_chunk=7, mode=mode)
    try:
        ids = [srv.submit(s, STEPS) for s in specs]
        max_running = _drain(srv, cap=4)
        assert max_running >= 2, "no two cases ran together"
        for rid, (f, t), spec in zip(ids, ref, specs):
            r = srv.poll(rid)
            assert r["state"] == ibm.REQ_DONE and r["status"] == 0, r
            assert r["steps_done"] == STEPS
            _same(r, f, t, mode, spec)
            assert r["submit_s"] <= r["start_s"] <= r["finish_s"]
        st = srv.stats()
        if mode & ibm.SERVE_BATCHED:
            assert st["group_steps"] > 0 and st["group_graphs"] > 0
            assert (st["autotune_runs"] > 0) == bool(mode & ibm.SERVE_AUTOTUNE)
        else:
            assert st["group_steps"] == 0
    finally:
        srv.close()


def test_batched_groups_against_oracle(orc):
    """Batched results against the FP64 oracle (not only against the case alone): one explicit group with a
    static, an oscillating, a free (Eq. 10) and a supersonic body, and one dual-time group at low Mach."""
    P = W.PREC_FP32_BULK
    cyl, dom = W.cylinder(256), (-8.0, 24.0, -8.0, 8.0)
    explicit = [W.case_spec(cyl, 128, 64, dom, 0.3, 100.0, W.FAR, precision=P, name="static"),
                W.case_spec(cyl, 128, 64, dom, 0.3, 100.0, W.FAR, motion=W.MOTION_SIN, amp=(0.0, 0.2), freq=0.16,
                            precision=P, name="osc"),
                _coupled(160, 64),
                W.wedge_m2_re1e4(128, 64, precision=P)]
    dual = [W.case_spec(cyl, 128, 64, dom, 0.01, 100.0, W.FAR, time_scheme=W.TIME_DUAL, dt_phys=0.125,
                        subiters=10, precision=P, name="dual_cyl"),
            W.case_spec(W.naca00xx(0.12, 400, 5.0), 160, 80, (-1.0, 3.0, -1.0, 1.0), 0.01, 500.0, W.FAR,
                        time_scheme=W.TIME_DUAL, dt_phys=0.025, subiters=10, precision=P, name="dual_naca")]
    jobs = [(s, 40) for s in explicit] + [(s, 4) for s in dual]
    srv = ibm.Server(max_active=8, steps_per_chunk=10)
    try:
        ids = [srv.submit(s, n) for s, n in jobs]
        assert _drain(srv, cap=8) == len(jobs)
        st = srv.stats()
        assert st["group_graphs"] >= 2 and st["group_steps"] > 0  # an explicit and a dual-time group
        for rid, (spec, n) in zip(ids, jobs):
            r = srv.poll(rid)
            assert r["state"] == ibm.REQ_DONE and r["status"] == 0 and r["steps_done"] == n, r
            o = orc.Case(dict(spec, precision=W.PREC_FP64))
            o.step(n)
            fo = o.forces()
            d = np.abs(r["forces"][:2] - fo[:2])
            print("%s: batched Cd, Cl %s oracle %s" % (spec["name"], r["forces"][:2], fo[:2]))
            assert d.max() <= 1e-3, (spec["name"], d)
            assert abs(r["t"] - o.time()) <= 1e-5 * o.time(), spec["name"]
    finally:
        srv.close()


def test_tvd2_and_quadratic_requests_batch():
    """Explicit requests with the TVD-2 reconstruction and / or the quadratic IB reconstruction form groups of
    their own variant (the group kernel is compiled for each), and give what they give alone up to FP32 rounding;
    a dual-time request with either runs on its own stream, bit for bit."""
    base = [s for s in _specs(6) if s["time_scheme"] == W.TIME_RK3][:3]
    odd = [dict(base[0], scheme=W.SCHEME_TVD2, name="tvd2"), dict(base[1], ib_interp=W.INTERP_QUADRATIC, name="quad"),
           dict(base[2], scheme=W.SCHEME_TVD2, ib_interp=W.INTERP_QUADRATIC, name="tvd2_quad")]
    dual_q = dict(W.case_spec(W.cylinder(128), 96, 48, (-3.0, 9.0, -3.0, 3.0), 0.01, 40.0, W.FAR,
                              time_scheme=W.TIME_DUAL, dt_phys=0.125, subiters=5, precision=W.PREC_FP32_BULK),
                  ib_interp=W.INTERP_QUADRATIC, name="dual_quad")
    # the variant requests alone in a server: they run in groups
    ref = [_alone(s, STEPS) for s in odd]
    srv = ibm.Server(max_active=6, steps_per_chunk=7)
    try:
        ids = [srv.submit(s, STEPS) for s in odd]
        _drain(srv, cap=6)
        assert srv.stats()["group_graphs"] >= len(odd)  # one group per variant
        for rid, (f, t), spec in zip(ids, ref, odd):
            r = srv.poll(rid)
            assert r["state"] == ibm.REQ_DONE and r["status"] == 0, r
            _same(r, f, t, MODES[0], spec)
    finally:
        srv.close()
    # mixed with plain requests and a dual-time request with the quadratic reconstruction
    specs = base + odd + [dual_q]
    ref = [_alone(s, 4 if s is dual_q else STEPS) for s in specs]
    srv = ibm.Server(max_active=8, steps_per_chunk=7)
    try:
        ids = [srv.submit(s, 4 if s is dual_q else STEPS) for s in specs]
        _drain(srv, cap=8)
        for rid, (f, t), spec in zip(ids, ref, specs):
            r = srv.poll(rid)
            assert r["state"] == ibm.REQ_DONE and r["status"] == 0, r
            if spec is dual_q:  # on its own stream: the kernels of the case alone
                np.testing.assert_array_equal(r["forces"], f)
                assert r["t"] == t
            else:
                _same(r, f, t, MODES[0], spec)
    finally:
        srv.close()


def test_batched_group_of_many_cases():
    """A full group (more cases than one group holds) of equal-size requests, batched vs alone."""
    # 64x64 and 128x64 grids share a size class: 30 cases fill one group and start a second
    specs = [s for s in (r["spec"] for r in W.serving_mix(600))
             if (s["nx"], s["ny"]) in ((64, 64), (128, 64)) and s["time_scheme"] == W.TIME_RK3]
    specs = specs[:30]
    assert len(specs) == 30
    ref = [_alone(s, 11) for s in specs]
    srv = ibm.Server(max_active=30, steps_per_chunk=4)
    try:
        ids = [srv.submit(s, 11) for s in specs]
        assert _drain(srv, cap=30) == 30
        for rid, (f, t), spec in zip(ids, ref, specs):
            r = srv.poll(rid)
            assert r["state"] == ibm.REQ_DONE, r
            _same(r, f, t, MODES[0], spec)
        st = srv.stats()
        assert st["group_graphs"] >= 2  # 30 cases of one size class need two groups
    finally:
        srv.close()


@pytest.mark.parametrize("mode", [MODES[0], 0])
def test_requests_arriving_while_others_run(mode):
    """Requests submitted between passes of the loop join the running cases."""
    specs = _specs(8)
    ref = [_alone(s, STEPS) for s in specs]
    srv = ibm.Server(max_active=3, steps_per_chunk=5, mode=mode)
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
        for rid, (f, t), spec in zip(ids, ref, specs):
            r = srv.poll(rid)
            assert r["state"] == ibm.REQ_DONE, r
            _same(r, f, t, mode, spec)
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
