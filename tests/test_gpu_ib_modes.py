"""IB nodes advanced by the flux update (IB_ADVANCE) on the GPU against the FP64 oracle, through the C ABI: a
cylinder in a Mach 2 stream, where only this treatment holds the bow shock, an oscillating cylinder whose cells
change role, and dual time at low Mach.  Bar: tags exact, FP64 state and forces within 1e-10 (the dual-time bar at
low Mach), FP32-bulk forces within 1e-3."""
import numpy as np
import pytest

from paper_1912_11908_gb300 import workloads as W

pytestmark = pytest.mark.gpu


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


def _state_err(a, b, tags):
    live = tags != 1
    return float(np.max(np.abs(a - b)[:, live] / np.maximum(1.0, np.abs(b)[:, live])))


@pytest.mark.parametrize("name,spec_fn,nsteps", [
    ("cylinder_M2_192x96", lambda: W.stationary_cylinder_supersonic(2.0, 192, 96, length=24.0, height=12.0,
                                                                    upstream=6.0, ib_mode=W.IB_ADVANCE), 150),
    ("osc_cylinder_128x64", lambda: dict(W.oscillating_cylinder_m02_re185(128, 64, ib_mode=W.IB_ADVANCE),
                                         amp=(0.0, 0.6), freq=0.5), 60),
])
def test_ib_advance_fp64_parity(ibm, orc, name, spec_fn, nsteps):
    spec = spec_fn()
    g, o = ibm.Case(spec), orc.Case(spec)
    g.step(nsteps)
    o.step(nsteps)
    np.testing.assert_array_equal(g.tags(), o.tags())
    err = _state_err(g.state(), o.state(), o.tags())
    assert err <= 1e-10, err
    np.testing.assert_allclose(g.forces(), o.forces(), rtol=0, atol=1e-10)


@pytest.mark.parametrize("name,spec_fn,nsteps", [
    ("cylinder_M2_192x96", lambda p: W.stationary_cylinder_supersonic(2.0, 192, 96, length=24.0, height=12.0,
                                                                     upstream=6.0, ib_mode=W.IB_ADVANCE,
                                                                     precision=p), 150),
    ("osc_cylinder_128x64", lambda p: dict(W.oscillating_cylinder_m02_re185(128, 64, ib_mode=W.IB_ADVANCE,
                                                                            precision=p),
                                           amp=(0.0, 0.6), freq=0.5), 60),
])
def test_ib_advance_fp32_bulk_vs_fp64_oracle(ibm, orc, name, spec_fn, nsteps):
    """FP32-bulk body tiles skip the IB rebuild and advance IB nodes: forces within 1e-3 of the FP64 oracle,
    state within 1e-3 of the deviation scale."""
    g, o = ibm.Case(spec_fn(W.PREC_FP32_BULK)), orc.Case(spec_fn(W.PREC_FP64))
    g.step(nsteps)
    o.step(nsteps)
    np.testing.assert_array_equal(g.tags(), o.tags())
    fg, fo = g.forces(), o.forces()
    assert abs(fg[0] - fo[0]) <= 1e-3 and abs(fg[1] - fo[1]) <= 1e-3, (fg, fo)
    a, b = g.state(), o.state()
    live = (o.tags() == 0) | (o.tags() == 2)
    for k in range(4):
        ref = b[k][live]
        dev = np.abs(ref - np.median(ref)).max() + 1e-300
        assert np.abs(a[k][live] - ref).max() <= 1e-3 * dev, k


@pytest.mark.parametrize("M", [0.01, 0.001])
def test_ib_advance_dual_time(ibm, orc, M):
    """Dual time with IB nodes advanced by the point-implicit update (FP64: state within the dual-time bar;
    FP32-bulk: forces within 1e-3 of the FP64 oracle)."""
    from flowmetrics import fp64_bar
    spec = W.case_spec(W.cylinder(128), 96, 48, (-3.0, 9.0, -3.0, 3.0), M, 40.0, W.FAR, time_scheme=W.TIME_DUAL,
                       dt_phys=0.125, subiters=10, ib_mode=W.IB_ADVANCE)
    o = orc.Case(spec)
    o.step(4)
    g = ibm.Case(spec)
    g.step(4)
    np.testing.assert_array_equal(g.tags(), o.tags())
    err, bar = _state_err(g.state(), o.state(), o.tags()), fp64_bar(orc, spec, 4)
    assert err <= bar, (err, bar)
    g32 = ibm.Case(dict(spec, precision=W.PREC_FP32_BULK))
    g32.step(4)
    d = np.abs(g32.forces()[:2] - o.forces()[:2])
    print("IB_ADVANCE dual time M %g: FP64 state %.2e (bar %.2e); FP32-bulk |dCd|, |dCl| %s" % (M, err, bar, d))
    assert d.max() <= 1e-3, d
