"""3-D immersed-boundary pre-processing on the GPU against the FP64 oracle (Sec. 3.2, Sec. 4.1-4.2; Appendix A's
sphere of 1200 triangles in a 40^3 cube).

Bar: node tags, the ordered IB / G1 / G2 / G3 lists and every listed node's closest-feature record (closest point,
pseudo-normal, feature kind) bit for bit.  The oracle sees the lattice nodes the library uses,
lo + (index + 1/2) (hi - lo) / n, built here with the same binary64 operations.
"""
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


def _lattice(n, lo, hi):
    ax = [lo[a] + (np.arange(n[a]) + 0.5) * ((hi[a] - lo[a]) / n[a]) for a in range(3)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)


def _check(ibm, orc, verts, tris, n, lo, hi):
    b = ibm.Body3D(verts, tris)
    b.classify(n, lo, hi)
    tags = b.tags()
    counts = b.counts()
    nodes = b.nodes()
    rec = b.closest()
    b.close()
    pts = _lattice(n, lo, hi)
    solid = orc.classify_points_3d(verts, tris, pts).reshape(n[2], n[1], n[0])
    tags_o = orc.tags_3d(solid)
    np.testing.assert_array_equal(tags, tags_o)
    flat = tags_o.ravel()
    lists = [np.nonzero(flat == t)[0] for t in (2, 3, 4, 5)]
    np.testing.assert_array_equal(counts, [len(x) for x in lists])
    np.testing.assert_array_equal(nodes, np.concatenate(lists))
    cp, nrm, kind = orc.closest_3d(verts, tris, pts[nodes])
    np.testing.assert_array_equal(rec["node"], nodes)
    np.testing.assert_array_equal(rec["kind"], kind)
    assert rec["cp"].tobytes() == cp.tobytes(), np.abs(rec["cp"] - cp).max()
    assert rec["n"].tobytes() == nrm.tobytes(), np.abs(rec["n"] - nrm).max()
    return counts, np.bincount(kind, minlength=3)


def test_sphere_in_cube_appendix_a(ibm, orc):
    """Appendix A: a 1200-triangle sphere of radius 0.35 in the 40^3 lattice over the unit cube."""
    verts, tris = W.uv_sphere(21, 30, 0.35, (0.5, 0.5, 0.5))
    counts, kinds = _check(ibm, orc, verts, tris, (40, 40, 40), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    print("sphere in 40^3: IB/G1/G2/G3 %s, closest face/edge/vertex %s" % (counts.tolist(), kinds.tolist()))
    assert counts.min() > 500 and kinds[0] > 0 and kinds[1] > 0


def test_grid_aligned_boxes(ibm, orc):
    """Boxes whose faces, edges and corners lie on lattice planes and lines (rays through face diagonals, box
    edges and corners; nodes on the surface) and a ragged, non-cubic lattice."""
    for (blo, bhi), n, lo, hi in [
            (((0.25, 0.25, 0.25), (0.75, 0.75, 0.75)), (9, 9, 9), (-0.0625,) * 3, (1.0625,) * 3),
            (((0.125, 0.375, 0.25), (0.875, 0.625, 0.5)), (17, 13, 11), (-0.03125,) * 3,
             (1.03125, 0.78125, 0.65625)),
            (((-0.5, -0.25, 0.0), (0.5, 0.75, 0.25)), (33, 29, 21), (-1.03125, -0.78125, -0.53125),
             (1.03125, 1.03125, 0.78125))]:
        verts, tris = W.box_mesh(blo, bhi)
        counts, kinds = _check(ibm, orc, verts, tris, n, lo, hi)
        assert counts[0] > 0 and kinds[2] > 0


def test_rotated_box_and_offset_sphere(ibm, orc):
    """A box turned about an oblique axis and a sphere off the lattice's symmetry planes, on lattices of
    several waves of nodes."""
    verts, tris = W.box_mesh((-0.3, -0.2, -0.25), (0.3, 0.2, 0.25))
    ax = np.array([1.0, 2.0, 3.0]) / np.sqrt(14.0)
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    Rm = np.eye(3) + np.sin(0.7) * K + (1 - np.cos(0.7)) * K @ K
    _check(ibm, orc, verts @ Rm.T + 0.5, tris, (48, 40, 36), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    verts, tris = W.uv_sphere(21, 30, 0.3, (0.47, 0.52, 0.49))
    _check(ibm, orc, verts, tris, (64, 64, 64), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))


def test_reclassify_other_lattice_and_errors(ibm, orc):
    """One body classified on two lattices in a row (buffers re-sized), and the error paths."""
    verts, tris = W.uv_sphere(21, 30, 0.35, (0.5, 0.5, 0.5))
    b = ibm.Body3D(verts, tris)
    b.classify((40, 40, 40), (0.0,) * 3, (1.0,) * 3)
    b.classify((24, 30, 20), (0.0,) * 3, (1.0,) * 3)
    pts = _lattice((24, 30, 20), (0.0,) * 3, (1.0,) * 3)
    solid = orc.classify_points_3d(verts, tris, pts).reshape(20, 30, 24)
    np.testing.assert_array_equal(b.tags(), orc.tags_3d(solid))
    with pytest.raises(ibm.IbmError):
        b.classify((0, 4, 4), (0.0,) * 3, (1.0,) * 3)
    b.close()
    with pytest.raises(ibm.IbmError):
        ibm.Body3D(verts, np.array([[0, 1, 2], [0, 1, 999], [1, 2, 3], [0, 2, 3]]))
