"""The 3-D flow solver on the GPU (ibm_case3d_*) against the FP64 3-D oracle.

Bars: tags, list counts and every field of every stencil bit for bit (the stencil kernel evaluates the oracle's
formulas in the same IEEE basic operations, without contraction); the state within 1e-10 relative to each
variable's range after the steps (the residual kernels contract to FMA and divide through reciprocals: a few
ulps per stage, grown by the flow's sensitivity, as in 2-D); time and dt within 1e-13 relative; forces within
1e-9 relative to their magnitude (a fixed-order tree against the oracle's compensated sum).
"""
import math

import numpy as np
import pytest

from paper_1912_11908_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FS, OUT, PER = W.BC_FREESTREAM, W.BC_OUTFLOW, W.BC_PERIODIC


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


def _state_error(g, o, tags):
    live = tags != 1  # every node the solver writes (solid nodes stay at the free stream on both sides)
    err = 0.0
    for v in range(5):
        scale = max(np.abs(o[v][live]).max(), 1e-300)
        if v in (1, 2, 3):
            scale = max(scale, np.abs(o[0][live]).max())  # momentum components measured against rho U_ref
        err = max(err, np.abs(g[v][live] - o[v][live]).max() / scale)
    return err


def _sphere(n=(40, 32, 32), lo=(-1.5, -1.6, -1.6), hi=(2.5, 1.6, 1.6), **kw):
    verts, tris = W.uv_sphere(radius=0.5)
    return W.case3d_spec(verts, tris, n, lo, hi, 0.3, 100.0, W.FAR3D, ref_area=math.pi * 0.25, **kw)


def _compare_geometry(g, o):
    np.testing.assert_array_equal(g.tags(), o.tags())
    gs, os_ = g.stencils(), o.stencils()
    assert gs.shape == os_.shape
    np.testing.assert_array_equal(g.counts(), [(os_["kind"] == k).sum() for k in range(4)])
    for f in os_.dtype.names:
        np.testing.assert_array_equal(gs[f], os_[f], err_msg=f)


def test_sphere_geometry_bit_exact(ibm, orc):
    spec = _sphere()
    g, o = ibm.Case3D(spec), orc.Case3D(spec)
    assert o.classify() == 0
    _compare_geometry(g, o)
    c = g.counts()
    assert c.min() > 50 and (g.stencils()["mask"] == 255).mean() > 0.7


@pytest.mark.parametrize("nsteps", [1, 12])
def test_sphere_flow_parity(ibm, orc, nsteps):
    spec = _sphere()
    g, o = ibm.Case3D(spec), orc.Case3D(spec)
    g.step(nsteps)
    o.step(nsteps)
    tg, to = g.time(), np.array([o.time(), o.last_dt()])
    np.testing.assert_allclose(tg, to, rtol=1e-13)
    e = _state_error(g.state(), o.state(), o.tags())
    print("3-D sphere, %d steps: state %.2e" % (nsteps, e))
    assert e <= 1e-10, e
    fg, fo = g.forces(), o.forces()
    print("forces GPU %s oracle %s" % (fg[:3], fo[:3]))
    np.testing.assert_allclose(fg, fo, rtol=0, atol=1e-9 * np.abs(fo).max())
    assert np.abs(fo[0]) > 1e-3  # the drag has built up
    assert g.launches() > 0


def test_box_body_oblique_flow(ibm, orc):
    """Sharp edges and corners (edge and vertex pseudo-normals, Eq. 2-3), flow oblique to every axis, outflow on
    three sides and a ragged grid (no size a multiple of the block)."""
    verts, tris = W.box_mesh((-0.3, -0.25, -0.35), (0.35, 0.3, 0.25))
    spec = W.case3d_spec(verts, tris, (29, 23, 27), (-1.0, -0.9, -1.1), (1.9, 1.4, 1.6), 0.5, 200.0,
                         (FS, OUT, FS, OUT, FS, OUT), uinf=(0.8, 0.3, -0.4), ref_area=0.5)
    g, o = ibm.Case3D(spec), orc.Case3D(spec)
    assert o.classify() == 0
    _compare_geometry(g, o)
    assert {0, 1} <= set(np.unique(g.stencils()["region"]))  # face and edge pseudo-normals
    g.step(8)
    o.step(8)
    e = _state_error(g.state(), o.state(), o.tags())
    assert e <= 1e-10, e
    fo = o.forces()
    np.testing.assert_allclose(g.forces(), fo, rtol=0, atol=1e-9 * np.abs(fo).max())


@pytest.mark.parametrize("plane", ["xy", "xz", "yz"])
def test_no_body_halos_every_side(ibm, orc, plane):
    """No body: a smooth perturbation in a box with a different boundary condition on each pair of sides
    (free stream / outflow / periodic, rotated through the axes), viscous, against the oracle."""
    n = {"xy": (18, 14, 11), "xz": (11, 18, 14), "yz": (14, 11, 18)}[plane]
    bcs = {"xy": (FS, OUT, FS, FS, PER, PER), "xz": (PER, PER, FS, OUT, OUT, OUT),
           "yz": (OUT, OUT, PER, PER, FS, OUT)}[plane]
    spec = W.case3d_spec(None, None, n, (0, 0, 0), (1.0, 0.8, 0.9), 0.5, 50.0, bcs, uinf=(0.6, 0.2, -0.3))
    rng = np.random.default_rng(3)
    z, y, x = np.meshgrid(*[(np.arange(k) + 0.5) / k for k in n[::-1]], indexing="ij")
    g_, pinf = 1.4, 1.0 / (1.4 * 0.25)
    a = rng.uniform(1, 2, 6)
    r = 1.0 + 0.05 * np.sin(2 * np.pi * (a[0] * x + a[1] * y)) * np.cos(2 * np.pi * a[2] * z)
    u = 0.6 + 0.1 * np.cos(2 * np.pi * a[3] * y)
    v = 0.2 + 0.1 * np.sin(2 * np.pi * a[4] * z)
    w = -0.3 + 0.1 * np.sin(2 * np.pi * a[5] * x)
    p = pinf * (1.0 + 0.03 * np.cos(2 * np.pi * (x + z)))
    U = np.stack([r, r * u, r * v, r * w, p / (g_ - 1.0) + 0.5 * r * (u * u + v * v + w * w)])
    g, o = ibm.Case3D(spec), orc.Case3D(spec)
    g.set_state(U)
    o.set_state(U)
    g.step(6)
    o.step(6)
    e = _state_error(g.state(), o.state(), o.tags())
    assert e <= 1e-10, e
    np.testing.assert_allclose(g.time(), [o.time(), o.last_dt()], rtol=1e-13)


def test_full_size_sphere_one_step(ibm, orc):
    """The benchmark's 192 x 96 x 96 sphere case: geometry bit for bit and one step against the oracle."""
    spec = W.sphere_m03_re100()
    g, o = ibm.Case3D(spec), orc.Case3D(spec)
    assert o.classify() == 0
    _compare_geometry(g, o)
    g.step(1)
    o.step(1)
    e = _state_error(g.state(), o.state(), o.tags())
    assert e <= 1e-10, e
    fo = o.forces()
    np.testing.assert_allclose(g.forces(), fo, rtol=0, atol=1e-9 * np.abs(fo).max())


def test_full_size_sphere_fp32_bulk(ibm, orc):
    """The benchmark's launch configuration (FP32-bulk, 192 x 96 x 96): two steps against the FP64 oracle."""
    spec = W.sphere_m03_re100()
    g, o = ibm.Case3D(dict(spec, precision=W.PREC_FP32_BULK)), orc.Case3D(spec)
    g.step(2)
    o.step(2)
    e = _state_error(g.state(), o.state(), o.tags())
    d = np.abs(g.forces()[:3] - o.forces()[:3])
    assert e <= 1e-4, e
    assert d.max() <= 1e-3, d


@pytest.mark.parametrize("precision", [W.PREC_FP64, W.PREC_FP32_BULK])
def test_degenerate_sizes(ibm, orc, precision):
    """A body smaller than the spacing that holds no node (empty lists; it is stepped as free flow, and its
    force probes see the free stream), and the smallest grid (4 cells per axis, a ragged single block)."""
    verts, tris = W.uv_sphere(radius=0.01, center=(0.013, 0.011, 0.012))
    spec = W.case3d_spec(verts, tris, (20, 10, 10), (-1, -0.5, -0.5), (1, 0.5, 0.5), 0.3, 100.0, W.FAR3D,
                         precision=precision)
    g, o = ibm.Case3D(spec), orc.Case3D(spec)
    assert o.classify() == 0 and (o.tags() == 0).all()
    np.testing.assert_array_equal(g.counts(), [0, 0, 0, 0])
    g.step(3)
    o.step(3)
    assert _state_error(g.state(), o.state(), o.tags()) <= (1e-10 if precision == W.PREC_FP64 else 1e-4)
    spec = W.case3d_spec(None, None, (4, 4, 4), (0, 0, 0), (1, 1, 1), 0.5, 50.0, (PER,) * 6, uinf=(0.3, 0.2, 0.1),
                         precision=precision)
    rng = np.random.default_rng(5)
    U = np.stack([np.ones((4, 4, 4)), 0.3 + 0.01 * rng.standard_normal((4, 4, 4)),
                  0.2 * np.ones((4, 4, 4)), 0.1 * np.ones((4, 4, 4)), np.zeros((4, 4, 4))])
    U[4] = (1.0 / (1.4 * 0.25)) / 0.4 + 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0]
    g, o = ibm.Case3D(spec), orc.Case3D(spec)
    g.set_state(U)
    o.set_state(U)
    g.step(2)
    o.step(2)
    assert _state_error(g.state(), o.state(), o.tags()) <= (1e-10 if precision == W.PREC_FP64 else 1e-4)


def test_quiescent_sphere_stays_at_rest(ibm):
    verts, tris = W.uv_sphere(radius=0.5)
    spec = W.case3d_spec(verts, tris, (24, 24, 24), (-1, -1, -1), (1, 1, 1), 0.3, 100.0, (FS,) * 6,
                         uinf=(0.0, 0.0, 0.0), dt_fixed=1e-3)
    g = ibm.Case3D(spec)
    g.step(3)
    U = g.state()
    live = g.tags() != 1
    assert np.abs(U[1:4][:, live]).max() < 1e-12
    assert np.abs(U[0][live] - 1.0).max() < 1e-13


@pytest.mark.parametrize("body", ["sphere", "box"])
def test_fp32_bulk_against_the_fp64_oracle(ibm, orc, body):
    """FP32-bulk fluxes (perturbation form) with FP64 stage accumulation: forces within 1e-3 of the FP64
    oracle's (the FP32-bulk bar of the 2-D solver), state within 1e-4 of each variable's range, geometry
    unchanged."""
    if body == "sphere":
        spec, n = _sphere(), 12
    else:
        verts, tris = W.box_mesh((-0.3, -0.25, -0.35), (0.35, 0.3, 0.25))
        spec = W.case3d_spec(verts, tris, (29, 23, 27), (-1.0, -0.9, -1.1), (1.9, 1.4, 1.6), 0.5, 200.0,
                             (FS, OUT, FS, OUT, FS, OUT), uinf=(0.8, 0.3, -0.4), ref_area=0.5)
        n = 8
    g = ibm.Case3D(dict(spec, precision=W.PREC_FP32_BULK))
    o = orc.Case3D(spec)
    g.step(n)
    o.step(n)
    np.testing.assert_array_equal(g.tags(), o.tags())
    e = _state_error(g.state(), o.state(), o.tags())
    d = np.abs(g.forces()[:3] - o.forces()[:3])
    print("3-D %s FP32-bulk, %d steps: state %.2e, |dC| %s (oracle %s)" % (body, n, e, d, o.forces()[:3]))
    assert e <= 1e-4, e
    assert d.max() <= 1e-3, d
    np.testing.assert_allclose(g.time(), [o.time(), o.last_dt()], rtol=1e-6)


def test_fp32_bulk_keeps_rest_and_free_stream(ibm):
    """The perturbation form keeps p_inf and H_inf out of the FP32 sums: fluid at rest around the sphere stays
    at rest, and a uniform stream in a box without a body stays uniform, to FP64 rounding."""
    verts, tris = W.uv_sphere(radius=0.5)
    spec = W.case3d_spec(verts, tris, (24, 24, 24), (-1, -1, -1), (1, 1, 1), 0.3, 100.0, (FS,) * 6,
                         uinf=(0.0, 0.0, 0.0), dt_fixed=1e-3, precision=W.PREC_FP32_BULK)
    g = ibm.Case3D(spec)
    g.step(3)
    U = g.state()
    live = g.tags() != 1
    assert np.abs(U[1:4][:, live]).max() < 1e-12
    assert np.abs(U[0][live] - 1.0).max() < 1e-13
    spec = W.case3d_spec(None, None, (20, 12, 9), (0, 0, 0), (1, 1, 1), 0.8, 100.0, W.FAR3D, uinf=(0.9, -0.2, 0.3),
                         precision=W.PREC_FP32_BULK)
    g = ibm.Case3D(spec)
    U0 = g.state()
    g.step(4)
    np.testing.assert_allclose(g.state(), U0, rtol=1e-14, atol=1e-14)


def test_bad_probe_is_reported(ibm):
    """A body whose IB probes leave the domain (a box touching a domain side) is refused with IBM_ESTENCIL,
    not stepped with an empty stencil."""
    verts, tris = W.box_mesh((-0.5, -0.5, -0.5), (0.9, 0.5, 0.5))
    spec = W.case3d_spec(verts, tris, (16, 16, 16), (-1, -1, -1), (1, 1, 1), 0.3, 100.0, (FS,) * 6)
    with pytest.raises(ibm.IbmError) as ei:
        ibm.Case3D(spec)
    assert ei.value.status == ibm.IBM_ESTENCIL
