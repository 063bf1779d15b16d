"""The quadratic IB / ghost reconstruction (Sec. 4.5, Sec. 5; IBM_INTERP_QUADRATIC) on the GPU against the FP64
oracle.

Bars, those of the linear form: node tags, lists and stencils (second probe included) bit for bit with the
oracle (stencil coordinates of a moving body within 1e-12: its pose takes sin and cos); FP64 state within 1e-10
relative (four times the oracle's own one-ulp sensitivity where larger, dual time at low Mach); FP32-bulk forces
within 1e-3.  Low-speed cases, the flows the paper uses this form for.
"""
import numpy as np
import pytest

from paper_1912_11908_gb300 import workloads as W
from flowmetrics import fp64_bar, rel_state_error

pytestmark = pytest.mark.gpu

Q = dict(ib_interp=W.INTERP_QUADRATIC)


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
    "cylinder": (W.cylinder_m02_re40(96, 48, **Q), 100),
    "osc_cylinder": (W.oscillating_cylinder_m02_re185(160, 80, **Q), 80),
    "naca_sharp_te": (dict(W.naca0012_a5_m0001(192, 96, time_scheme=W.TIME_RK3, **Q), mach=0.3,
                           domain=(-0.5, 1.5, -0.5, 0.5)), 60),
    "cylinder_ib_advance": (W.cylinder_m02_re40(96, 48, ib_mode=W.IB_ADVANCE, **Q), 100),
    "cylinder_tvd2": (W.cylinder_m02_re40(96, 48, scheme=W.SCHEME_TVD2, **Q), 100),
}


def _compare_stencils(g, o, moving):
    np.testing.assert_array_equal(g.tags(), o.tags())
    gs, os_ = g.stencils(), np.concatenate([o.stencils(k) for k in range(4)])
    for f in ("cell", "mask", "region", "i0", "j0", "maskb", "i0b", "j0b", "nstepb"):
        np.testing.assert_array_equal(gs[f], os_[f], err_msg=f)
    for f in ("xi_probe", "xi_probe2", "w", "wb"):
        if moving:  # the pose takes sin / cos, whose last bits differ between the two math libraries
            np.testing.assert_allclose(gs[f], os_[f], rtol=0, atol=1e-12, err_msg=f)
        else:
            np.testing.assert_array_equal(gs[f], os_[f], err_msg=f)
    assert (gs["maskb"] != 0).mean() > 0.9  # the second probe found a square almost everywhere


@pytest.mark.parametrize("name", sorted(CASES))
def test_quadratic_fp64_parity(ibm, orc, name):
    spec, n = CASES[name]
    g, o = ibm.Case(spec), orc.Case(spec)
    for _ in range(2):
        g.step(n // 2)
        o.step(n // 2)
        _compare_stencils(g, o, spec["motion"] != W.MOTION_STATIC)
    e = rel_state_error(g.state(), o.state(), o.tags())
    print("quadratic %s FP64 after %d steps: state %.2e" % (name, n, e))
    assert e <= 1e-10, e
    np.testing.assert_allclose(g.forces(), o.forces(), rtol=1e-8, atol=1e-9)


def _dual():
    return W.case_spec(W.cylinder(128), 96, 48, (-3.0, 9.0, -3.0, 3.0), 0.01, 40.0, W.FAR, time_scheme=W.TIME_DUAL,
                       dt_phys=0.125, subiters=10, **Q)


def test_quadratic_dual_time_parity(ibm, orc):
    spec = _dual()
    g, o = ibm.Case(spec), orc.Case(spec)
    g.step(4)
    o.step(4)
    _compare_stencils(g, o, False)
    e, bar = rel_state_error(g.state(), o.state(), o.tags()), fp64_bar(orc, spec, 4)
    print("quadratic dual time M 0.01 FP64: state %.2e (bar %.2e)" % (e, bar))
    assert e <= bar, (e, bar)


@pytest.mark.parametrize("name", sorted(CASES) + ["dual"])
def test_quadratic_fp32_bulk_forces(ibm, orc, name):
    spec, n = (_dual(), 4) if name == "dual" else CASES[name]
    g = ibm.Case(dict(spec, precision=W.PREC_FP32_BULK))
    o = orc.Case(spec)
    g.step(n)
    o.step(n)
    np.testing.assert_array_equal(g.tags(), o.tags())
    d = np.abs(g.forces()[:2] - o.forces()[:2])
    print("quadratic %s FP32-bulk: |dCd|, |dCl| %s (oracle %s)" % (name, d, o.forces()[:2]))
    assert d.max() <= 1e-3, d


@pytest.mark.parametrize("precision", [W.PREC_FP64, W.PREC_FP32_BULK])
def test_quadratic_option_reaches_the_kernels(ibm, precision):
    """The two forms give different flows (the option is not dropped on the way to the kernels), and the second
    probe is only computed in the quadratic form."""
    spec, n = CASES["cylinder"]
    a = ibm.Case(dict(spec, precision=precision))
    b = ibm.Case(dict(spec, precision=precision, ib_interp=W.INTERP_LINEAR))
    a.step(n)
    b.step(n)
    assert np.abs(a.forces()[0] - b.forces()[0]) > 1e-5
    assert (b.stencils()["maskb"] == 0).all() and (a.stencils()["maskb"] != 0).any()
