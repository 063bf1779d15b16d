"""Pins of the oracle's two treatments of IB nodes.

IB_REBUILD rebuilds the fluid-side IB nodes from their probes every stage
(Sec. 4.4-4.6); IB_ADVANCE advances them by the flux update like fluid nodes
and imposes the wall through the rebuilt ghost layers alone (Sec. 5's field
extension).  The pins: both keep the exact solutions (gas at rest around a
sharp body, a body carried by a uniform stream), and in a supersonic stream
the stagnation pressure in front of a cylinder must reach the Rayleigh pitot
value of the free-stream Mach number.  IB_REBUILD does so at M = 1.2 but not at
M = 2, where the first fluid node ahead of the stagnation point stays
supersonic and the rebuilt IB node behind it discards what the upwind flux
carries in; IB_ADVANCE does so at both.
"""
import numpy as np
import pytest

from paper_1912_11908_gb300 import workloads as W


def _pitot(M, g=1.4):
    """Stagnation pressure behind a normal shock over the free-stream static pressure (Rayleigh)."""
    return ((g + 1) * M * M / 2) ** (g / (g - 1)) / ((2 * g * M * M - (g - 1)) / (g + 1)) ** (1 / (g - 1))


def _max_pressure_ratio(orc, M, mode):
    spec = W.stationary_cylinder_supersonic(M, 192, 96, length=24.0, height=12.0, upstream=6.0, ib_mode=mode)
    c = orc.Case(spec)
    while c.time() < 6.0:
        c.step(50)
    U = c.state()
    r = U[0]
    p = (spec["gamma"] - 1.0) * (U[3] - 0.5 * (U[1] ** 2 + U[2] ** 2) / r)
    t = c.tags()
    live = (t == 0) | (t == 2)  # fluid and IB nodes
    return p[live].max() * spec["gamma"] * M * M  # over p_inf = 1 / (gamma M^2)


@pytest.mark.parametrize("M,mode", [(1.2, W.IB_REBUILD), (1.2, W.IB_ADVANCE), (2.0, W.IB_ADVANCE)])
def test_stagnation_pressure_reaches_the_pitot_value(orc, M, mode):
    """Cylinder at D/8 in a stream at M, Re 300, t = 6: the largest pressure (the stagnation point) within 8% of
    the pitot value (5.64 p_inf at M 2; measured 1.007 of it with IB_ADVANCE, 0.21 with IB_REBUILD)."""
    ratio = _max_pressure_ratio(orc, M, mode) / _pitot(M)
    assert abs(ratio - 1.0) <= 0.08, ratio


def test_advance_mode_keeps_gas_at_rest_around_a_sharp_body(orc):
    spec = W.case_spec(W.naca00xx(0.12, 200, 10.0), 96, 48, (-0.5, 1.5, -0.5, 0.5), 0.3, 500.0, W.FAR,
                       uinf=(0.0, 0.0), ib_mode=W.IB_ADVANCE)
    c = orc.Case(spec)
    U0 = c.state()
    c.step(100)
    U1 = c.state()
    live = c.tags() != 1
    for k in range(4):
        assert np.abs(U1[k] - U0[k])[live].max() <= 1e-12 * max(1.0, np.abs(U0[k]).max()), k


def test_advance_mode_keeps_a_body_carried_by_the_stream(orc):
    spec = W.case_spec(W.cylinder(64, 1.0), 96, 48, (-2.0, 6.0, -2.0, 2.0), 0.5, 100.0, W.FAR,
                       motion=W.MOTION_CONST, vel=(1.0, 0.0), ib_mode=W.IB_ADVANCE)
    c = orc.Case(spec)
    U0 = c.state()
    c.step(60)
    assert c.time() > 0.4
    U1 = c.state()
    live = c.tags() != 1
    for k in range(4):
        assert np.abs(U1[k] - U0[k])[live].max() <= 1e-12 * max(1.0, np.abs(U0[k]).max()), k
