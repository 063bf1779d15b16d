"""Dual time stepping on the GPU (FP64) against the FP64 oracle.

BDF2 physical time, preconditioned point-implicit pseudo time in three stages per sub-iteration, FP64 4x4 solve per
cell (Sec. 2).  Bar: state within 1e-10 relative after several physical steps; tags / stencils as for RK3.
"""
import math

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
    err = _err(g.state(), o.state(), o.tags())
    assert err <= 1e-10, err
    np.testing.assert_allclose(g.forces(), o.forces(), rtol=1e-8, atol=1e-8)


def test_dual_naca_sharp_te_parity(ibm, orc):
    spec = W.naca0012_a5_m0001(256, 128, subiters=6)
    spec = dict(spec, domain=(-0.5, 1.5, -0.5, 0.5), dt_phys=0.5 * 2.0 / 256)
    g, o = ibm.Case(spec), orc.Case(spec)
    g.step(4)
    o.step(4)
    np.testing.assert_array_equal(g.tags(), o.tags())
    err = _err(g.state(), o.state(), o.tags())
    assert err <= 1e-10, err


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
    err = _err(g.state(), o.state(), np.zeros((8, nx), np.uint8))
    assert err <= 1e-10, err
