"""Dual time stepping on the GPU (FP64 and FP32-bulk) against the FP64 oracle.

BDF2 physical time, preconditioned point-implicit pseudo time in three stages per sub-iteration, FP64 4x4 solve per
cell (Sec. 2).  Bar: FP64 state within 1e-10 relative after several physical steps, or within four times the
oracle's own conditioning floor where that is larger (see ulp_floor); tags / stencils as for RK3.
"""
import math

import numpy as np
import pytest

from paper_1912_11908_gb300 import workloads as W
from flowmetrics import fp64_bar

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


def _err(a, b, tags):
    live = tags != 1
    return float(np.max(np.abs(a - b)[:, live] / np.maximum(1.0, np.abs(b)[:, live])))


@pytest.mark.parametrize("M", [0.01, 0.001])
def test_dual_cylinder_parity(ibm, orc, M):
    nx, ny = 96, 48
    spec = W.case_spec(W.cylinder(128), nx, ny, (-3.0, 9.0, -3.0, 3.0), M, 40.0, W.FAR, time_scheme=W.TIME_DUAL,
                       dt_phys=0.5 * 12.0 / nx, subiters=10)
    g, o = ibm.Case(spec), orc.Case(spec)
    g.step(6)
    o.step(6)
    assert abs(g.time()[0] - o.time()) < 1e-12
    err, bar = _err(g.state(), o.state(), o.tags()), fp64_bar(orc, spec, 6)
    print("dual cylinder M %g: FP64 state %.2e (bar %.2e)" % (M, err, bar))
    assert err <= bar, (err, bar)
    np.testing.assert_allclose(g.forces(), o.forces(), rtol=1e-8, atol=max(1e-8, bar))


def test_dual_naca_sharp_te_parity(ibm, orc):
    spec = W.naca0012_a5_m0001(256, 128, subiters=6)
    spec = dict(spec, domain=(-0.5, 1.5, -0.5, 0.5), dt_phys=0.5 * 2.0 / 256)
    g, o = ibm.Case(spec), orc.Case(spec)
    g.step(4)
    o.step(4)
    np.testing.assert_array_equal(g.tags(), o.tags())
    err, bar = _err(g.state(), o.state(), o.tags()), fp64_bar(orc, spec, 4)
    print("dual NACA sharp TE: FP64 state %.2e (bar %.2e)" % (err, bar))
    assert err <= bar, (err, bar)


def test_dual_entropy_wave_periodic(ibm, orc):
    nx = 64
    dx = 1.0 / nx
    M = 0.001
    spec = W.case_spec(None, nx, 8, (0.0, 1.0, 0.0, 8 * dx), M, 0.0, W.PERIODIC, time_scheme=W.TIME_DUAL,
                       dt_phys=0.5 * dx, subiters=30, uinf=(1.0, 0.0))
    g, o = ibm.Case(spec), orc.Case(spec)
    X = np.tile((np.arange(nx) + 0.5) * dx, (8, 1))
    pinf = 1.0 / (1.4 * M * M)
    r = 1.0 + 0.01 * np.sin(2 * math.pi * X)
    U = np.stack([r, r, 0 * r, pinf / 0.4 + 0.5 * r])
    g.set_state(U)
    o.set_state(U)
    g.step(5)
    o.step(5)
    err, bar = _err(g.state(), o.state(), np.zeros((8, nx), np.uint8)), fp64_bar(orc, spec, 5, U)
    print("dual entropy wave: FP64 state %.2e (bar %.2e)" % (err, bar))
    assert err <= bar, (err, bar)


# ---- FP32-bulk dual time: FP32 perturbation residual, FP64 point-implicit update and iterates ----

def _pressure(U, M, gamma=1.4):
    r, mx, my, E = U
    return (gamma - 1.0) * (E - 0.5 * (mx * mx + my * my) / r) - 1.0 / (gamma * M * M)


def _bulk_vs_oracle(ibm, orc, spec, nsteps):
    sb = dict(spec, precision=W.PREC_FP32_BULK)
    g, o = ibm.Case(sb), orc.Case(spec)
    g.step(nsteps)
    o.step(nsteps)
    assert abs(g.time()[0] - o.time()) < 1e-12
    live = o.tags() == 0
    a, b = g.state(), o.state()
    pa, pb = _pressure(a, spec["mach"])[live], _pressure(b, spec["mach"])[live]
    dp = float(np.abs(pa - pb).max() / np.abs(pb - np.median(pb)).max())
    du = float(max(np.abs(a[k] / a[0] - b[k] / b[0])[live].max() for k in (1, 2)))
    df = np.abs(g.forces()[:2] - o.forces()[:2])
    print("bulk dual %s: p' rel %.3e, velocity %.3e, |dCd|,|dCl| %s" % (spec["name"] or spec["mach"], dp, du, df))
    return dp, du, df


# Tolerances.  The FP32 residual carries face velocities to FP32 rounding (~6e-8 of U) and pressure perturbations
# to ~6e-8 of their own size (the perturbation form keeps p_inf = 1/(gamma M^2) out of every FP32 sum).  The
# preconditioned LDFSS dissipation scales velocity differences by rho c' with c' of the order of the reference
# velocity U_r = max(|V|, U_ref, nu/dn) -- independent of M -- so the rounding floor of the residual is ~1e-7 of
# the dynamic scale at any Mach number; the pseudo-time coefficients (FP32) change the path of the sub-iterations
# but not their fixed point.  Bounds: |dCd|, |dCl| <= 1e-4 at M = 0.01 and the configuration's 1e-3 at
# M = 0.001 (a coarse 8-cells-per-diameter cylinder, 10 sub-iterations: the pseudo iteration is far from converged,
# so FP32 rounding of the path is not damped out).
@pytest.mark.parametrize("M,force_tol", [(0.01, 1e-4), (0.001, 1e-3)])
def test_bulk_dual_cylinder_vs_fp64_oracle(ibm, orc, M, force_tol):
    nx, ny = 96, 48
    spec = W.case_spec(W.cylinder(128), nx, ny, (-3.0, 9.0, -3.0, 3.0), M, 40.0, W.FAR, time_scheme=W.TIME_DUAL,
                       dt_phys=0.5 * 12.0 / nx, subiters=10)
    dp, du, df = _bulk_vs_oracle(ibm, orc, spec, 6)
    assert df.max() <= force_tol, df
    assert du <= 1e-3, du
    assert dp <= 1e-2, dp


def test_bulk_dual_naca_m0001_vs_fp64_oracle(ibm, orc):
    spec = W.naca0012_a5_m0001(256, 128, subiters=10)
    spec = dict(spec, domain=(-0.5, 1.5, -0.5, 0.5), dt_phys=0.5 * 2.0 / 256)
    dp, du, df = _bulk_vs_oracle(ibm, orc, spec, 4)
    assert df.max() <= 1e-3, df
    assert du <= 1e-3, du
    assert dp <= 1e-2, dp


def test_bulk_dual_entropy_wave_keeps_pressure_uniform(ibm, orc):
    """An entropy (density) wave in a uniform stream at M = 0.001: the density wave and the (small) pressure
    disturbance match the FP64 oracle."""
    nx = 64
    dx = 1.0 / nx
    M = 0.001
    spec = W.case_spec(None, nx, 8, (0.0, 1.0, 0.0, 8 * dx), M, 0.0, W.PERIODIC, time_scheme=W.TIME_DUAL,
                       dt_phys=0.5 * dx, subiters=30, uinf=(1.0, 0.0), precision=W.PREC_FP32_BULK)
    g, o = ibm.Case(spec), orc.Case(dict(spec, precision=W.PREC_FP64))
    X = np.tile((np.arange(nx) + 0.5) * dx, (8, 1))
    pinf = 1.0 / (1.4 * M * M)
    r = 1.0 + 0.01 * np.sin(2 * math.pi * X)
    U = np.stack([r, r, 0 * r, pinf / 0.4 + 0.5 * r])
    g.set_state(U)
    o.set_state(U)
    g.step(5)
    o.step(5)
    a, b = g.state(), o.state()
    drho = float(np.abs(a[0] - b[0]).max() / 0.01)
    pa, pb = _pressure(a, M), _pressure(b, M)
    dpp = float(np.abs(pa - pb).max())  # in units of the dynamic pressure rho U^2 = 1
    print("bulk dual entropy wave: density rel %.3e, max |p'| %.3e (oracle %.3e), |dp'| %.3e"
          % (drho, np.abs(pa).max(), np.abs(pb).max(), dpp))
    assert drho <= 1e-4, drho
    assert np.abs(pa).max() < 0.05  # the scheme's own bound (oracle pin)
    assert dpp <= 1e-2, dpp


def test_bulk_dual_launch_forms(ibm):
    """Pseudo stages as one launch each, chained by programmatic dependent launch, give bit for bit what the
    same kernel gives launched plainly; the two-stream plain / body kernels (compiled separately) agree to FP32
    rounding."""
    spec = W.case_spec(W.cylinder(128), 96, 48, (-3.0, 9.0, -3.0, 3.0), 0.01, 40.0, W.FAR, time_scheme=W.TIME_DUAL,
                       dt_phys=0.5 * 12.0 / 96, subiters=10, precision=W.PREC_FP32_BULK)
    runs = {}
    for mode in (0, 1, 2):
        c = ibm.Case(spec)
        c.stage_launches(mode)
        c.step(4)
        assert c.stage_launch() == mode
        runs[mode] = (c.state(), c.forces())
    np.testing.assert_array_equal(runs[2][0], runs[1][0])
    np.testing.assert_array_equal(runs[2][1], runs[1][1])
    np.testing.assert_allclose(runs[2][1], runs[0][1], rtol=1e-5, atol=1e-5 * np.abs(runs[0][1]).max())


def test_integer_bit_conversions_match_hardware(ibm):
    """The dual-time update converts FP32 <-> FP64 on the integer bits of the IEEE 754 formats (the FP64 pipe
    bounds it): every binary32 value but the flushed subnormals, and 2^30 binary64 patterns including exact
    rounding ties and exponents outside the binary32 range, convert exactly as the hardware does."""
    n, bad = ibm.check_float_conversions()
    assert n == (1 << 32) - 2 * ((1 << 23) - 1) + (1 << 30)
    assert bad == 0
