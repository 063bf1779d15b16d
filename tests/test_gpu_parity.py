"""GPU (sm_103a) library vs the FP64 CPU oracle, through the C ABI.

Bar: bit-exact tags, IB / ghost lists and interpolation stencils; FP64 state
within 1e-10 relative L-infinity after 100 steps; forces within 1e-10.  Sizes
span several 16x16 tiles with ragged tails.
"""
import math

import numpy as np
import pytest

from paper_1912_11908_gb300 import workloads as W

pytestmark = pytest.mark.gpu

STATE_RTOL = 1e-10


@pytest.fixture(scope="module")
def ibm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1912_11908_gb300 import _build, ibm as mod
    _build.build()
    mod.lib()
    return mod


def _oracle_stencils(o):
    return np.concatenate([o.stencils(k) for k in range(4)])


def _state_err(a, b, tags):
    live = tags != 1
    return float(np.max(np.abs(a - b)[:, live] / np.maximum(1.0, np.abs(b)[:, live])))


GEOMETRY_CASES = {
    "cylinder_160x80": lambda: W.cylinder_m02_re40(),
    "cylinder_ragged_150x70": lambda: W.cylinder_m02_re40(150, 70),
    "wedge_192x96": lambda: W.wedge_m2_re1e4(192, 96),
    "wedge_768x384": lambda: W.wedge_m2_re1e4(768, 384),
    "naca_a5_330x170": lambda: W.case_spec(W.naca00xx(0.12, 400, 5.0), 330, 170, (-0.6, 1.6, -0.55, 0.55), 0.5,
                                           1000.0, W.FAR),
    "naca_a5_2048x1024": lambda: W.naca0012_a5_m0001(time_scheme=W.TIME_RK3),
    "osc_cylinder_1024x512": lambda: W.oscillating_cylinder_m02_re185(),
}


@pytest.mark.parametrize("name", sorted(GEOMETRY_CASES))
def test_tags_lists_stencils_bit_exact(ibm, orc, name):
    spec = GEOMETRY_CASES[name]()
    g = ibm.Case(spec)
    o = orc.Case(spec)
    g.classify()
    o.classify()
    np.testing.assert_array_equal(g.tags(), o.tags())
    counts = g.counts()
    assert [int(c) for c in counts] == [len(o.stencils(k)) for k in range(4)]
    gs, os_ = g.stencils(), _oracle_stencils(o)
    assert gs.dtype.itemsize == os_.dtype.itemsize == 176
    assert gs.tobytes() == os_.tobytes()


def test_random_polygons_bit_exact(ibm, orc):
    rng = np.random.default_rng(21)
    done = 0
    while done < 5:
        verts = W.random_polygon(rng, int(rng.integers(5, 30)), rmin=0.5, rmax=0.9)
        spec = W.case_spec(verts, 97, 83, (-1.2, 1.3, -1.1, 1.05), 0.5, 200.0, W.FAR)
        o = orc.Case(spec)
        if o.classify() != 0:
            continue  # a spike too thin for any valid interpolation corner (IBM_ESTENCIL by design)
        done += 1
        g = ibm.Case(spec)
        g.classify()
        np.testing.assert_array_equal(g.tags(), o.tags())
        assert g.stencils().tobytes() == _oracle_stencils(o).tobytes()


def _run_pair(ibm, orc, spec, nsteps, chunks=1):
    g, o = ibm.Case(spec), orc.Case(spec)
    for _ in range(chunks):
        g.step(nsteps // chunks)
        o.step(nsteps // chunks)
    return g, o


@pytest.mark.parametrize("name,spec_fn,nsteps", [
    ("cylinder_M0.2_Re40_160x80", lambda: W.cylinder_m02_re40(), 100),
    ("cylinder_ragged_150x70", lambda: W.cylinder_m02_re40(150, 70), 100),
    ("wedge_M2_192x96", lambda: W.wedge_m2_re1e4(192, 96), 100),
    ("naca_sharp_te_M0.5", lambda: W.case_spec(W.naca00xx(0.12, 400, 5.0), 200, 104, (-0.6, 1.6, -0.55, 0.55),
                                               0.5, 1000.0, W.FAR), 100),
    ("periodic_box_no_body", lambda: W.case_spec(None, 64, 40, (0.0, 1.0, 0.0, 0.625), 0.4, 100.0, W.PERIODIC,
                                                 uinf=(0.3, 0.1)), 100),
])
def test_state_parity_fp64(ibm, orc, name, spec_fn, nsteps):
    spec = spec_fn()
    g, o = ibm.Case(spec), orc.Case(spec)
    if len(spec["verts"]) == 0:
        # perturb the uniform state so the no-body box has something to do
        ny, nx = spec["ny"], spec["nx"]
        X, Y = np.meshgrid((np.arange(nx) + 0.5) / nx, (np.arange(ny) + 0.5) / ny)
        r = 1.0 + 0.1 * np.sin(2 * math.pi * X) * np.cos(2 * math.pi * Y)
        U = np.stack([r, r * 0.3, r * 0.1, 1.0 / (1.4 * 0.16) / 0.4 + 0.5 * r * 0.1 + 0 * X])
        g.set_state(U)
        o.set_state(U)
    g.step(nsteps)
    o.step(nsteps)
    tg, to = g.time(), o.time()
    assert abs(tg[0] - to) <= 1e-12 * max(1.0, to)
    err = _state_err(g.state(), o.state(), o.tags())
    assert err <= STATE_RTOL, err
    if len(spec["verts"]):
        np.testing.assert_allclose(g.forces(), o.forces(), rtol=0, atol=1e-10)


def test_moving_body_parity(ibm, orc):
    """Oscillating cylinder: re-classification every step on the GPU and in the oracle."""
    spec = W.oscillating_cylinder_m02_re185(128, 64)
    spec = dict(spec, amp=(0.0, 0.6), freq=0.5)  # large motion: cells change role within the run
    g, o = ibm.Case(spec), orc.Case(spec)
    for _ in range(5):
        g.step(20)
        o.step(20)
        np.testing.assert_array_equal(g.tags(), o.tags())
        gs, os_ = g.stencils(), _oracle_stencils(o)
        np.testing.assert_array_equal(gs["cell"], os_["cell"])
        np.testing.assert_array_equal(gs["mask"], os_["mask"])
        for f in ("bx", "by", "xi_node", "xi_probe", "nx", "ny"):
            np.testing.assert_allclose(gs[f], os_[f], rtol=0, atol=1e-12)
    err = _state_err(g.state(), o.state(), o.tags())
    assert err <= STATE_RTOL, err
    np.testing.assert_allclose(g.forces(), o.forces(), rtol=0, atol=1e-10)


def test_quiescent_and_translating_free_stream(ibm):
    for spec in (W.case_spec(W.naca00xx(0.12, 200, 10.0), 96, 48, (-0.5, 1.5, -0.5, 0.5), 0.3, 500.0, W.FAR,
                             uinf=(0.0, 0.0)),
                 W.case_spec(W.cylinder(64, 1.0), 96, 48, (-2.0, 6.0, -2.0, 2.0), 0.5, 100.0, W.FAR,
                             motion=W.MOTION_CONST, vel=(1.0, 0.0))):
        g = ibm.Case(spec)
        U0 = g.state()
        g.step(60)
        U1 = g.state()
        live = g.tags() != 1
        for k in range(4):
            assert np.abs(U1[k] - U0[k])[live].max() <= 1e-12 * max(1.0, np.abs(U0[k]).max())


def test_full_size_wedge_768x384_parity(ibm, orc):
    """Full-size workload in the benchmark's launch configuration: 3 steps, every cell compared."""
    spec = W.wedge_m2_re1e4()
    g, o = ibm.Case(spec), orc.Case(spec)
    g.step(3)
    o.step(3)
    err = _state_err(g.state(), o.state(), o.tags())
    assert err <= STATE_RTOL, err


def test_set_get_state_roundtrip_and_device_copy(ibm):
    import torch
    spec = W.cylinder_m02_re40(100, 52)
    g = ibm.Case(spec)
    g.step(5)
    a = g.state()
    t = torch.empty((4, 52, 100), dtype=torch.float64, device="cuda")
    g.state_to_device(t)
    np.testing.assert_array_equal(t.cpu().numpy(), a)
    h = ibm.Case(spec)
    h.set_state(a)
    np.testing.assert_array_equal(h.state(), a)


def test_errors_are_reported(ibm):
    spec = W.cylinder_m02_re40(64, 32)
    bad = dict(spec, nx=4)
    with pytest.raises(ibm.IbmError) as e:
        ibm.Case(bad)
    assert e.value.status == ibm.IBM_EINVAL
    g = ibm.Case(spec)
    with pytest.raises(ibm.IbmError):
        g.step(-1)
