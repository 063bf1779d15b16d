"""Pitching motion on the GPU (Sec. 7.2: NACA0012 pitching about mid-chord) against the FP64 oracle.

The pose turns the reference airfoil and its normals about the pivot at every step; each IB / ghost node's wall
velocity and acceleration are those of the rigid rotation at its boundary point, as are the force probes'.
Bars: tags and lists exact at every checkpoint, stencil coordinates within 1e-12 (the pose takes sin and cos of
the body angle, whose last bits differ between the two math libraries), FP64 state within 1e-10 relative (four
times the oracle's own one-ulp sensitivity at low Mach where larger), FP32-bulk forces within 1e-3.
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


def _explicit(**kw):
    # 1 chord airfoil, pivot at mid-chord, fast pitching: the body turns by about 7 degrees in 120 steps, the
    # trailing edge moving at a quarter of the sound speed
    spec = W.pitching_naca0012(160, 120, freq=2.0, mach=0.3, re=500.0, time_scheme=W.TIME_RK3, **kw)
    return dict(spec, domain=(-0.5, 1.5, -0.75, 0.75))


def _dual(**kw):
    spec = W.pitching_naca0012(128, 96, freq=2.0, re=500.0, subiters=10, **kw)
    return dict(spec, domain=(-0.5, 1.5, -0.75, 0.75), dt_phys=0.5 * 2.0 / 128)


def _compare_geometry(g, o):
    np.testing.assert_array_equal(g.tags(), o.tags())
    gs, os_ = g.stencils(), np.concatenate([o.stencils(k) for k in range(4)])
    np.testing.assert_array_equal(gs["cell"], os_["cell"])
    np.testing.assert_array_equal(gs["mask"], os_["mask"])
    np.testing.assert_array_equal(gs["region"], os_["region"])
    for f in ("bx", "by", "xi_node", "xi_probe", "nx", "ny"):
        np.testing.assert_allclose(gs[f], os_[f], rtol=0, atol=1e-12)


def test_pitching_explicit_fp64_parity(ibm, orc):
    spec = _explicit()
    g, o = ibm.Case(spec), orc.Case(spec)
    for _ in range(4):
        g.step(30)
        o.step(30)
        _compare_geometry(g, o)
    e = rel_state_error(g.state(), o.state(), o.tags())
    print("pitching RK3 FP64 after 120 steps (t = %.3f): state %.2e" % (o.time(), e))
    assert e <= 1e-10, e
    np.testing.assert_allclose(g.forces(), o.forces(), rtol=1e-8, atol=1e-9)
    cpg, cfg = g.surface()
    cpo, cfo = o.surface()
    np.testing.assert_allclose(cpg, cpo, rtol=1e-8, atol=1e-9)
    np.testing.assert_allclose(cfg, cfo, rtol=1e-8, atol=1e-9)


def test_pitching_dual_time_fp64_parity(ibm, orc):
    spec = _dual()
    g, o = ibm.Case(spec), orc.Case(spec)
    for _ in range(3):
        g.step(1)
        o.step(1)
        _compare_geometry(g, o)
    e, bar = rel_state_error(g.state(), o.state(), o.tags()), fp64_bar(orc, spec, 3)
    print("pitching dual time M %g FP64 after 3 steps: state %.2e (bar %.2e)" % (spec["mach"], e, bar))
    assert e <= bar, (e, bar)


@pytest.mark.parametrize("kind", ["explicit", "dual"])
def test_pitching_fp32_bulk_forces(ibm, orc, kind):
    spec, n = (_explicit(), 120) if kind == "explicit" else (_dual(), 3)
    g = ibm.Case(dict(spec, precision=W.PREC_FP32_BULK))
    o = orc.Case(spec)
    g.step(n)
    o.step(n)
    np.testing.assert_array_equal(g.tags(), o.tags())
    d = np.abs(g.forces()[:2] - o.forces()[:2])
    print("pitching %s FP32-bulk: |dCd|, |dCl| %s (oracle %s)" % (kind, d, o.forces()[:2]))
    assert d.max() <= 1e-3, d


def test_pitching_moves_the_wall(ibm):
    """The option reaches the kernels: a pitching airfoil and the same airfoil held at its mean incidence part
    ways (the rotation changes the tags and the flow)."""
    a = ibm.Case(_explicit())
    b = ibm.Case(dict(_explicit(), motion=W.MOTION_STATIC, verts=W.naca00xx(0.12, 400, 0.0)))
    a.step(120)
    b.step(120)
    assert (a.tags() != b.tags()).sum() > 10
