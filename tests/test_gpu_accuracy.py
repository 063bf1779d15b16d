"""Accuracy of every configuration's results at the configuration's own size: the GPU paths against the FP64
oracle (Cd, Cl, surface Cp, state) and the wedge's oblique shock against the theta-beta-M relation.

Bars: FP64 state within 1e-10 relative (at M = 0.001: four times the oracle's own sensitivity to a one-ulp
change of its initial state, where that is larger); FP32-bulk |dCd|, |dCl| <= 1e-3; the steady shock between
theta-beta-M at the geometric wedge angle and at that angle plus the boundary layer's displacement slope.  Each
test prints what it measured.
"""
import math

import numpy as np
import pytest

from paper_1912_11908_gb300 import workloads as W
from flowmetrics import deviation_error, fp64_bar, theta_from_beta, theta_from_ratio, wedge_shock

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


def _rel64(a, b, tags):
    live = tags != 1
    return float(np.max(np.abs(a - b)[:, live] / np.maximum(1.0, np.abs(b)[:, live])))


def _freestream(spec):
    g, M = spec["gamma"], spec["mach"]
    u, v = spec["uinf"]
    return np.array([1.0, u, v, 1.0 / (g * M * M) / (g - 1.0) + 0.5 * (u * u + v * v)])[:, None, None]


def _bulk_report(name, g32, o, spec):
    f32, fo = g32.forces(), o.forces()
    cp32, _ = g32.surface()
    cpo, _ = o.surface()
    ok = np.isfinite(cpo) & np.isfinite(cp32)
    live = o.tags() == 0
    dev = deviation_error(g32.state(), o.state(), live, _freestream(spec))
    rep = dict(dcd=abs(f32[0] - fo[0]), dcl=abs(f32[1] - fo[1]), cp_linf=float(np.abs(cp32 - cpo)[ok].max()),
               cp_range=float(np.ptp(cpo[ok])), state_dev=max(dev))
    print("%s FP32-bulk vs oracle: |dCd| %.2e |dCl| %.2e  surface Cp Linf %.2e (range %.3f)  state / deviation %.2e"
          "  (oracle Cd %.5f Cl %.5f)" % (name, rep["dcd"], rep["dcl"], rep["cp_linf"], rep["cp_range"],
                                          rep["state_dev"], fo[0], fo[1]))
    return rep


def test_wedge_768x384_vs_oracle(ibm, orc):
    """Configuration wedge 15 deg, M 2, Re 1e4, 768 x 384: 200 RK3 steps, FP64 and FP32-bulk."""
    spec = W.wedge_m2_re1e4()
    o = orc.Case(spec)
    o.step(200)
    g64 = ibm.Case(spec)
    g64.step(200)
    e = _rel64(g64.state(), o.state(), o.tags())
    print("wedge 768x384 FP64 GPU vs oracle after 200 steps: state %.2e" % e)
    assert e <= 1e-10, e
    np.testing.assert_allclose(g64.forces(), o.forces(), rtol=1e-8, atol=1e-9)
    g32 = ibm.Case(dict(spec, precision=W.PREC_FP32_BULK))
    g32.step(200)
    r = _bulk_report("wedge 768x384", g32, o, spec)
    assert r["dcd"] <= 1e-3 and r["dcl"] <= 1e-3, r
    assert r["cp_linf"] <= 1e-2 * r["cp_range"], r


def test_wedge_oblique_shock(ibm):
    """The wedge's attached oblique shock at steady state (t >= 4; the impulsively started flow is still forming
    it at the configuration's 2000 steps, whose values are printed), in both precisions.  theta-beta-M is the
    inviscid relation; at Re 1e4 the laminar boundary layer on the wedge face thickens the body the stream sees
    by its displacement slope, d(delta*)/dx = 0.86 C / sqrt(Re_x) with C ~ 2 for an adiabatic wall at the
    post-shock Mach 1.45, about 1 deg at mid-chord (Re_x ~ 9000).  Bar: the wedge angle for which theta-beta-M
    gives the measured shock angle, and the one that gives the measured pressure ratio, lie between the
    geometric 15 deg and 16.5 deg; FP32-bulk and FP64 agree within 0.1 deg and 0.2%.  (The angle is fitted to the
    shock's position over x = 0.45 ... 0.75: 0.1 deg is a tenth of a cell, dx = 4 / 768, of shock displacement
    across that 0.3 chord; the two precisions' roundings settle the captured shock at slightly different sub-cell
    positions, measured 0.05-0.06 deg apart.)"""
    res = {}
    for precision in (W.PREC_FP32_BULK, W.PREC_FP64):
        spec = W.wedge_m2_re1e4(precision=precision)
        g = ibm.Case(spec)
        g.step(2000)
        b0, r0 = wedge_shock(g.state(), g.tags(), spec)
        t0 = g.time()[0]
        while g.time()[0] < 4.0:
            g.step(500)
        beta, ratio = wedge_shock(g.state(), g.tags(), spec)
        th_b, th_r = theta_from_beta(2.0, math.radians(beta)), theta_from_ratio(2.0, ratio)
        print("wedge 768x384 %s: after 2000 steps (t = %.3f) shock %.2f deg, p2/p1 %.4f; at t = %.3f shock %.2f deg,"
              " p2/p1 %.4f (theta-beta-M at 15 deg: 45.34, 2.1947): effective wedge %.2f deg from the angle, %.2f deg "
              "from the ratio" % ("FP32-bulk" if precision else "FP64", t0, b0, r0, g.time()[0], beta, ratio, th_b,
                                  th_r))
        assert 15.0 <= th_b <= 16.5 and 15.0 <= th_r <= 16.5, (th_b, th_r)
        res[precision] = (beta, ratio)
    (b32, r32), (b64, r64) = res[W.PREC_FP32_BULK], res[W.PREC_FP64]
    assert abs(b32 - b64) <= math.degrees(math.atan(0.1 * (4.0 / 768) / 0.3)) and abs(r32 / r64 - 1.0) <= 2e-3


def test_oscillating_cylinder_1024x512_vs_oracle(ibm, orc):
    """Configuration oscillating cylinder, M 0.2, Re 185, 1024 x 512, re-classified every step: Cd and Cl every
    40 steps over 200 steps against the oracle (FP32-bulk), and the FP64 state at the end."""
    spec = W.oscillating_cylinder_m02_re185()
    o = orc.Case(spec)
    g64 = ibm.Case(spec)
    g32 = ibm.Case(dict(spec, precision=W.PREC_FP32_BULK))
    worst = 0.0
    for _ in range(5):
        o.step(40)
        g64.step(40)
        g32.step(40)
        fo, f32 = o.forces(), g32.forces()
        worst = max(worst, abs(fo[0] - f32[0]), abs(fo[1] - f32[1]))
        np.testing.assert_allclose(g64.forces(), fo, rtol=1e-8, atol=1e-8)
    np.testing.assert_array_equal(g64.tags(), o.tags())
    e = _rel64(g64.state(), o.state(), o.tags())
    print("oscillating cylinder 1024x512 FP64 GPU vs oracle after 200 steps: state %.2e; FP32-bulk max |dC| over "
          "the window %.2e" % (e, worst))
    assert e <= 1e-10, e
    r = _bulk_report("oscillating cylinder 1024x512", g32, o, spec)
    assert worst <= 1e-3 and r["dcd"] <= 1e-3 and r["dcl"] <= 1e-3, (worst, r)


def test_naca_2048x1024_dual_m0001_vs_oracle(ibm, orc):
    """Configuration NACA0012 at 5 deg, M 0.001, Re 1000, 2048 x 1024, dual time with 30 sub-iterations: two
    physical steps, FP64 state and FP32-bulk forces and surface Cp."""
    spec = W.naca0012_a5_m0001()
    o = orc.Case(spec)
    o.step(2)
    g64 = ibm.Case(spec)
    g64.step(2)
    e, bar = _rel64(g64.state(), o.state(), o.tags()), fp64_bar(orc, spec, 2)
    print("NACA0012 2048x1024 dual FP64 GPU vs oracle after 2 physical steps: state %.2e (bar %.2e: the "
          "oracle's own 1-ulp sensitivity x 4)" % (e, bar))
    assert e <= bar, (e, bar)
    g32 = ibm.Case(dict(spec, precision=W.PREC_FP32_BULK))
    g32.step(2)
    r = _bulk_report("NACA0012 2048x1024 dual M 0.001", g32, o, spec)
    assert r["dcd"] <= 1e-3 and r["dcl"] <= 1e-3, r
    assert r["cp_linf"] <= 1e-2 * r["cp_range"], r


def test_cylinder_160x80_fp32_bulk_vs_oracle(ibm, orc):
    """Configuration cylinder M 0.2, Re 40, 160 x 80, 200 steps: FP32-bulk forces and surface Cp."""
    spec = W.cylinder_m02_re40()
    o = orc.Case(spec)
    o.step(200)
    g32 = ibm.Case(dict(spec, precision=W.PREC_FP32_BULK))
    g32.step(200)
    r = _bulk_report("cylinder 160x80", g32, o, spec)
    assert r["dcd"] <= 1e-3 and r["dcl"] <= 1e-3, r
    assert r["cp_linf"] <= 1e-2 * r["cp_range"], r


def test_surface_matches_forces_and_oracle(ibm, orc):
    """ibm_surface against the oracle's per-segment Cp and Cf (FP64, 1e-10), and its midpoint sums against
    ibm_forces' Cd."""
    spec = W.cylinder_m02_re40(80, 40)
    g, o = ibm.Case(spec), orc.Case(spec)
    g.step(30)
    o.step(30)
    cpg, cfg = g.surface()
    cpo, cfo = o.surface()
    np.testing.assert_allclose(cpg, cpo, rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(cfg, cfo, rtol=1e-9, atol=1e-10)
    v = spec["verts"]
    e = np.roll(v, -1, axis=0) - v
    L = np.linalg.norm(e, axis=1)
    t = e / L[:, None]
    n = np.stack([t[:, 1], -t[:, 0]], 1)
    cd = np.sum((-cpg * n[:, 0] + cfg * t[:, 0]) * L)
    assert abs(cd - g.forces()[0]) < 1e-9
