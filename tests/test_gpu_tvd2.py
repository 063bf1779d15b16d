"""The second-order TVD reconstruction (Sec. 2; MUSCL with the minmod limiter) on the GPU against the FP64 oracle.

Bar: FP64 state within 1e-10 relative (four times the oracle's own one-ulp sensitivity where larger, dual time at
low Mach), FP32-bulk forces within 1e-3 -- the bars of the WENO5 path.
"""
import numpy as np
import pytest

from paper_1912_11908_gb300 import workloads as W
from flowmetrics import fp64_bar, rel_state_error

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


CASES = {
    "cylinder": (W.cylinder_m02_re40(96, 48, scheme=W.SCHEME_TVD2), 100),
    "wedge_m2": (W.wedge_m2_re1e4(192, 96, scheme=W.SCHEME_TVD2), 100),
    "naca_sharp_te": (dict(W.naca0012_a5_m0001(192, 96, scheme=W.SCHEME_TVD2, time_scheme=W.TIME_RK3), mach=0.3,
                           domain=(-0.5, 1.5, -0.5, 0.5)), 60),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_tvd2_fp64_parity(ibm, orc, name):
    spec, n = CASES[name]
    g, o = ibm.Case(spec), orc.Case(spec)
    g.step(n)
    o.step(n)
    np.testing.assert_array_equal(g.tags(), o.tags())
    e = rel_state_error(g.state(), o.state(), o.tags())
    print("TVD-2 %s FP64 after %d steps: state %.2e" % (name, n, e))
    assert e <= 1e-10, e
    np.testing.assert_allclose(g.forces(), o.forces(), rtol=1e-8, atol=1e-9)


def test_tvd2_dual_time_parity(ibm, orc):
    spec = W.case_spec(W.cylinder(128), 96, 48, (-3.0, 9.0, -3.0, 3.0), 0.01, 40.0, W.FAR, time_scheme=W.TIME_DUAL,
                       dt_phys=0.125, subiters=10, scheme=W.SCHEME_TVD2)
    g, o = ibm.Case(spec), orc.Case(spec)
    g.step(4)
    o.step(4)
    e, bar = rel_state_error(g.state(), o.state(), o.tags()), fp64_bar(orc, spec, 4)
    print("TVD-2 dual time M 0.01 FP64: state %.2e (bar %.2e)" % (e, bar))
    assert e <= bar, (e, bar)


@pytest.mark.parametrize("name", sorted(CASES))
def test_tvd2_fp32_bulk_forces(ibm, orc, name):
    spec, n = CASES[name]
    g = ibm.Case(dict(spec, precision=W.PREC_FP32_BULK))
    o = orc.Case(spec)
    g.step(n)
    o.step(n)
    fg, fo = g.forces(), o.forces()
    d = np.abs(fg[:2] - fo[:2])
    print("TVD-2 %s FP32-bulk: |dCd|, |dCl| %s (oracle %s)" % (name, d, fo[:2]))
    assert d.max() <= 1e-3, d


def test_tvd2_differs_from_weno5(ibm):
    """The option reaches the kernels: the same case with the two reconstructions gives different states."""
    spec, n = CASES["wedge_m2"]
    a = ibm.Case(dict(spec, precision=W.PREC_FP32_BULK))
    b = ibm.Case(dict(spec, precision=W.PREC_FP32_BULK, scheme=W.SCHEME_WENO5))
    a.step(20)
    b.step(20)
    assert np.abs(a.state() - b.state()).max() > 1e-6
