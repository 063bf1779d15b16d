"""Body moving under the fluid force (Sec. 6, Eq. 10) on the GPU, through the C ABI: the shock-driven
cylinder of Sec. 8.2.6 on coarse grids against the FP64 oracle.

Bar: tags and lists exact at every checkpoint; FP64 state within 1e-10 and body displacement, velocity and
force within 1e-10; FP32-bulk forces within 1e-3 and body velocity within 1e-3 of its scale.
"""
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


def _state_err(a, b, tags):
    live = tags != 1
    return float(np.max(np.abs(a - b)[:, live] / np.maximum(1.0, np.abs(b)[:, live])))


@pytest.mark.parametrize("nx,ny", [(64, 64), (90, 74)])
def test_shock_driven_cylinder_fp64_parity(ibm, orc, nx, ny):
    spec = W.shock_driven_cylinder(nx, ny, density_ratio=2.0)
    U0 = W.shock_initial_state(spec)
    g, o = ibm.Case(spec), orc.Case(spec)
    g.set_state(U0)
    o.set_state(U0)
    for _ in range(6):
        g.step(25)
        o.step(25)
        np.testing.assert_array_equal(g.tags(), o.tags())
        np.testing.assert_allclose(g.body(), o.body(), rtol=1e-10, atol=1e-12)
    assert o.time() > 1.0 and o.body()[2] > 0.05  # the shock has passed and set the body moving
    err = _state_err(g.state(), o.state(), o.tags())
    assert err <= STATE_RTOL, err
    np.testing.assert_allclose(g.forces(), o.forces(), rtol=0, atol=1e-10)


def test_shock_driven_cylinder_fp32_bulk(ibm, orc):
    spec = W.shock_driven_cylinder(64, 64, density_ratio=2.0)
    U0 = W.shock_initial_state(spec)
    g = ibm.Case(dict(spec, precision=W.PREC_FP32_BULK))
    o = orc.Case(spec)
    g.set_state(U0)
    o.set_state(U0)
    for _ in range(6):
        g.step(25)
        o.step(25)
        np.testing.assert_array_equal(g.tags(), o.tags())
        fg, fo = g.forces(), o.forces()
        assert abs(fg[0] - fo[0]) <= 1e-3 and abs(fg[1] - fo[1]) <= 1e-3, (fg, fo)
    bg, bo = g.body(), o.body()
    assert abs(bg[2] - bo[2]) <= 1e-3 * abs(bo[2]) and abs(bg[0] - bo[0]) <= 1e-3 * abs(bo[0]), (bg, bo)


def test_coupled_motion_is_validated(ibm):
    spec = W.shock_driven_cylinder(64, 64)
    with pytest.raises(ibm.IbmError):
        ibm.Case(dict(spec, mass=0.0))
    with pytest.raises(ibm.IbmError):
        ibm.Case(dict(spec, time_scheme=W.TIME_DUAL, dt_phys=0.01))
