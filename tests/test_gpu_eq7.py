"""Supersonic moving-body pressure condition (Eq. 7) on the GPU, through the C ABI.

Bar: bit-exact stencils including the local curvature (IEEE geometry on both
sides) for a static body; the FP64 path within 1e-10 of the oracle while the
condition acts in every stage of a cylinder crossing the grid at M = 1.2 and 2; the FP32-bulk path
within the FP32-bulk bar (forces 1e-3, state 1e-3 of the deviation scale);
and the Galilean-invariance check of Sec. 8.2.3: the drag of the cylinder
moving through gas at rest against the drag of the same cylinder at rest in
the stream, at two resolutions.
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


def _small_moving(mach_d=1.2, **kw):
    # 12 x 4 diameters at D/10 (ragged against the 16 x 16 tiles), centre 2 diameters from the right side
    return W.moving_cylinder_supersonic(mach_d, 120, 40, length=12.0, height=4.0, start=2.0, **kw)


def test_curvature_stencils_bit_exact_on_nonconvex_body(ibm, orc):
    a, n = 0.25, 3000
    th = 2.0 * math.pi * np.arange(n) / n
    r = 1.0 + a * np.cos(3 * th)
    verts = np.stack([r * np.cos(th), r * np.sin(th)], 1)
    spec = W.case_spec(verts, 200, 200, (-1.5, 1.5, -1.5, 1.5), 0.5, 100.0, W.FAR)
    g, o = ibm.Case(spec), orc.Case(spec)
    g.classify()
    assert o.classify() == 0
    gs, os_ = g.stencils(), _oracle_stencils(o)
    assert (os_["curv"] < 0).any() and (os_["curv"] > 0).any()
    assert gs.tobytes() == os_.tobytes()


@pytest.mark.parametrize("mach_d", [1.2, 2.0])
def test_supersonic_moving_cylinder_fp64_parity(ibm, orc, mach_d):
    """Tags and lists exact at each checkpoint while the body crosses cells, stencil geometry and curvature to
    1e-12 (the pose follows t, whose time steps carry FMA-level differences); the state within 1e-10 and the
    forces within 1e-10 with the Eq. 7 term applied to every IB and ghost node."""
    spec = _small_moving(mach_d)
    g, o = ibm.Case(spec), orc.Case(spec)
    for _ in range(4):
        g.step(15)
        o.step(15)
        np.testing.assert_array_equal(g.tags(), o.tags())
        gs, os_ = g.stencils(), _oracle_stencils(o)
        np.testing.assert_array_equal(gs["cell"], os_["cell"])
        np.testing.assert_array_equal(gs["mask"], os_["mask"])
        for f in ("bx", "by", "xi_node", "xi_probe", "nx", "ny", "curv"):
            np.testing.assert_allclose(gs[f], os_[f], rtol=0, atol=1e-12)
    assert o.time() > 0.5  # several cells crossed
    err = _state_err(g.state(), o.state(), o.tags())
    assert err <= STATE_RTOL, err
    np.testing.assert_allclose(g.forces(), o.forces(), rtol=0, atol=1e-10)


def test_supersonic_moving_cylinder_fp32_bulk(ibm, orc):
    g = ibm.Case(_small_moving(precision=W.PREC_FP32_BULK))
    o = orc.Case(_small_moving())
    for _ in range(3):
        g.step(20)
        o.step(20)
        np.testing.assert_array_equal(g.tags(), o.tags())
        fg, fo = g.forces(), o.forces()
        assert abs(fg[0] - fo[0]) <= 1e-3 and abs(fg[1] - fo[1]) <= 1e-3, (fg, fo)
    a, b = g.state(), o.state()
    live = o.tags() == 0
    for k in range(4):
        ref = b[k][live]
        dev = np.abs(ref - np.median(ref)).max() + 1e-300
        assert np.abs(a[k][live] - ref).max() <= 1e-3 * dev, k


def _mean_drag(case, t_end, t_avg, chunk=50):
    """Drag coefficient averaged over samples every `chunk` steps in the last t_avg time units before t_end."""
    samples = []
    while True:
        case.step(chunk)
        t = case.time()[0]
        if t >= t_end - t_avg:
            samples.append(case.forces()[0])
        if t >= t_end:
            return float(np.mean(samples)), float(np.std(samples))


@pytest.mark.parametrize("mach_d,ib_mode,extrap_bound", [(1.2, W.IB_REBUILD, 0.01), (2.0, W.IB_ADVANCE, 0.02)])
def test_galilean_invariance_moving_vs_stationary(ibm, mach_d, ib_mode, extrap_bound):
    """Sec. 8.2.3, Re_D = 300: the mean drag over t = 24-30 of the cylinder moving through gas at rest (40 x 12
    diameters) against that of the cylinder at rest in the stream (24 x 12 diameters), at D/16 and D/32.  The
    wall conditions differ between the two by design: the moving body's carries the Eq. 7 gradient over the
    probe distance, the body at rest (Eq. 6) none, so the two drags differ by a first-order term in h.
    Measured with the oracle: M_D 1.2, -6.83% at D/16, -3.38% at D/32, extrapolated (2 d_32 - d_16) 0.07%;
    M_D 2.0 with IB nodes advanced by the flux update (the rebuilt nodes do not hold the bow shock there),
    -6.23% and -2.47%, extrapolated 1.3%.  Bounds: the difference shrinks like h (ratio <= 0.6) and its
    extrapolation to h = 0 is within 1% (M 1.2) or 2% (M 2)."""
    t_end, t_avg = 30.0, 6.0
    d = {}
    for res in (16, 32):
        mv = ibm.Case(W.moving_cylinder_supersonic(mach_d, 40 * res, 12 * res, length=40.0, height=12.0, start=4.0,
                                                   ib_mode=ib_mode))
        st = ibm.Case(W.stationary_cylinder_supersonic(mach_d, 24 * res, 12 * res, length=24.0, height=12.0,
                                                       upstream=6.0, ib_mode=ib_mode))
        cd_m, sd_m = _mean_drag(mv, t_end, t_avg)
        cd_s, sd_s = _mean_drag(st, t_end, t_avg)
        print("M_D=%g D/%d  Cd moving %.5f (+-%.5f)  stationary %.5f (+-%.5f)" % (mach_d, res, cd_m, sd_m, cd_s,
                                                                                  sd_s))
        assert 1.3 < cd_s < 1.8  # cylinder at M 1.2-2, Re 300: bow shock and wake
        d[res] = (cd_m - cd_s) / cd_s
        mv.close()
        st.close()
    assert abs(d[32]) <= 0.6 * abs(d[16]), d
    assert abs(2.0 * d[32] - d[16]) <= extrap_bound, d
