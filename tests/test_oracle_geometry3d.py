"""Pins of the oracle's 3-D node classification (Sec. 3.2: Moller-Trumbore ray casting against a closed
triangulated surface; Appendix A's sphere of 1200 triangles in a 40^3 cube).  The GPU library does not build
the 3-D path yet; these pins fix the oracle its kernels will be held to.

The reference is the winding number of the closed surface, the sum of the solid angles its triangles subtend
(van Oosterom and Strackee's closed form), an independent definition of inside: 1 inside, 0 outside.
"""
import numpy as np

from paper_1912_11908_gb300 import workloads as W


def _winding(verts, tris, pts, chunk=2048):
    a0, b0, c0 = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    out = np.empty(len(pts))
    for s in range(0, len(pts), chunk):
        p = pts[s:s + chunk, None, :]
        a, b, c = a0[None] - p, b0[None] - p, c0[None] - p
        la, lb, lc = (np.linalg.norm(x, axis=2) for x in (a, b, c))
        num = np.einsum("pti,pti->pt", a, np.cross(b, c))
        den = (la * lb * lc + np.einsum("pti,pti->pt", a, b) * lc + np.einsum("pti,pti->pt", a, c) * lb
               + np.einsum("pti,pti->pt", b, c) * la)
        out[s:s + chunk] = (2.0 * np.arctan2(num, den)).sum(axis=1) / (4.0 * np.pi)
    return out


def test_sphere_in_cube_matches_the_winding_number(orc):
    """Every node of the 40^3 grid over the unit cube against a 1200-triangle sphere of radius 0.35."""
    verts, tris = W.uv_sphere(21, 30, 0.35, (0.5, 0.5, 0.5))
    assert len(tris) == 1200
    g = (np.arange(40) + 0.5) / 40
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    solid = orc.classify_points_3d(verts, tris, pts)
    wind = _winding(verts, tris, pts)
    assert np.all(np.abs(wind - np.round(wind)) < 1e-6)  # no node on the surface
    np.testing.assert_array_equal(solid, (wind > 0.5).astype(np.uint8))
    # the inscribed polyhedron holds a little less than the ball's 4/3 pi 0.35^3 40^3 = 11,494 nodes
    assert 0.95 * 11494 < solid.sum() <= 11494


def test_rays_through_vertices_and_edges(orc):
    """Points whose +x ray passes exactly through mesh vertices or along edges (where one ray can count a
    crossing twice or not at all): the majority of three rays still agrees with the winding number."""
    verts, tris = W.uv_sphere(21, 30, 1.0)
    rng = np.random.default_rng(7)
    pick = rng.choice(len(verts), 200, replace=False)
    shifts = rng.uniform(0.05, 2.5, 200)
    pts = verts[pick] - np.stack([shifts, 0 * shifts, 0 * shifts], 1)  # +x ray hits the vertex exactly
    mids = 0.5 * (verts[tris[:100, 0]] + verts[tris[:100, 1]])  # edge midpoints, approached along -x
    pts = np.concatenate([pts, mids - np.array([0.3, 0.0, 0.0])])
    wind = _winding(verts, tris, pts)
    keep = np.abs(wind - np.round(wind)) < 1e-6
    assert keep.sum() > 250
    solid = orc.classify_points_3d(verts, tris, pts[keep])
    np.testing.assert_array_equal(solid, (wind[keep] > 0.5).astype(np.uint8))
    assert 0 < solid.sum() < keep.sum()  # both sides are exercised


def test_pseudo_normal_sign_matches_inside_near_sharp_edges(orc):
    """Angle-weighted vertex and edge pseudo-normals (Eq. 2, 3): near every face, edge and corner of a box and
    of the sphere, sign((X - C).n) < 0 exactly for the points inside (the property that makes the signed
    distance consistent at sharp features, Sec. 4.2)."""
    rng = np.random.default_rng(13)
    for verts, tris in (W.box_mesh((0.1, 0.2, 0.3), (0.9, 0.7, 1.1)), W.uv_sphere(21, 30, 0.5)):
        idx = rng.integers(0, len(verts), 600)
        pts = np.concatenate([verts[idx] + rng.normal(scale=0.05, size=(600, 3)),
                              verts[tris[rng.integers(0, len(tris), 600)]].mean(axis=1)
                              + rng.normal(scale=0.05, size=(600, 3))])
        cp, nrm, kind = orc.closest_3d(verts, tris, pts)
        wind = _winding(verts, tris, pts)
        d = np.einsum("pi,pi->p", pts - cp, nrm)
        ok = np.linalg.norm(pts - cp, axis=1) > 1e-9
        assert ok.sum() > 1100
        np.testing.assert_array_equal((d < 0)[ok], (wind > 0.5)[ok])
        assert set(np.unique(kind[ok])) == {0, 1, 2}  # faces, edges and vertices all exercised


def test_closest_point_against_dense_sampling(orc):
    verts, tris = W.uv_sphere(11, 16, 1.0)
    g = np.linspace(0.0, 1.0, 41)
    S, T = np.meshgrid(g, g)
    keep = S + T <= 1.0
    s, t = S[keep], T[keep]
    samples = np.concatenate([verts[f[0]] + s[:, None] * (verts[f[1]] - verts[f[0]])
                              + t[:, None] * (verts[f[2]] - verts[f[0]]) for f in tris])
    rng = np.random.default_rng(5)
    pts = rng.normal(size=(150, 3))
    pts *= rng.uniform(0.5, 1.5, (150, 1)) / np.linalg.norm(pts, axis=1, keepdims=True)
    cp, _, _ = orc.closest_3d(verts, tris, pts)
    dist = np.linalg.norm(pts - cp, axis=1)
    for k in range(len(pts)):
        dmin = np.min(np.linalg.norm(samples - pts[k], axis=1))
        assert dist[k] <= dmin + 1e-12
        assert dist[k] >= dmin - 0.02  # sampling resolution (edge length / 40)
        assert np.min(np.linalg.norm(samples - cp[k], axis=1)) < 0.02  # the point lies on the surface


def _tags_by_definition_3d(solid):
    """Tags written out from the definitions with array shifts: IB = fluid with a solid 6-neighbour; G_s = solid
    with a non-solid node s steps away along some axis and none closer."""
    nz, ny, nx = solid.shape
    pad = np.pad(solid, 3, constant_values=0).astype(bool)
    inner = (slice(3, 3 + nz), slice(3, 3 + ny), slice(3, 3 + nx))

    def shifted(s, axis):
        sl = [slice(3, 3 + nz), slice(3, 3 + ny), slice(3, 3 + nx)]
        sl[axis] = slice(3 + s, 3 + s + solid.shape[axis])
        return pad[tuple(sl)]

    # outside the lattice counts as neither solid (for IB) nor non-solid (for ghosts)
    valid = np.pad(np.ones_like(solid, bool), 3, constant_values=False)

    def in_lattice(s, axis):
        sl = [slice(3, 3 + nz), slice(3, 3 + ny), slice(3, 3 + nx)]
        sl[axis] = slice(3 + s, 3 + s + solid.shape[axis])
        return valid[tuple(sl)]

    s0 = pad[inner]
    tags = np.where(s0, 1, 0).astype(np.uint8)
    nb_solid = np.zeros_like(s0)
    for axis in range(3):
        for s in (1, -1):
            nb_solid |= shifted(s, axis) & in_lattice(s, axis)
    tags[~s0 & nb_solid] = 2
    done = ~s0
    for step in (1, 2, 3):
        hit = np.zeros_like(s0)
        for axis in range(3):
            for s in (step, -step):
                hit |= ~shifted(s, axis) & in_lattice(s, axis)
        new = s0 & ~done & hit
        tags[new] = 2 + step
        done |= new
    return tags


def test_tags_3d_by_definition(orc):
    verts, tris = W.uv_sphere(21, 30, 0.35, (0.5, 0.5, 0.5))
    g = (np.arange(40) + 0.5) / 40
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    solid = orc.classify_points_3d(verts, tris, pts).reshape(40, 40, 40)
    tags = orc.tags_3d(solid)
    np.testing.assert_array_equal(tags, _tags_by_definition_3d(solid))
    counts = np.bincount(tags.ravel(), minlength=6)
    assert all(counts[k] > 500 for k in (2, 3, 4, 5)), counts


def test_grid_aligned_box_meshes(orc):
    """Boxes whose faces, edges and corners lie on lattice planes and lines, so that the rays of most nodes pass
    exactly through triangle edges (the quad diagonals), box edges or corners.  Every strictly interior lattice
    node is solid and every exterior node fluid (nodes on the surface may fall either way): an edge or vertex
    crossing counted twice or missed flips a node here."""
    cases = [((0.25, 0.25, 0.25), (0.75, 0.75, 0.75), 8), ((0.25, 0.25, 0.25), (0.75, 0.75, 0.75), 32),
             ((0.125, 0.375, 0.25), (0.875, 0.625, 0.5), 16), ((-0.5, -0.25, 0.0), (0.5, 0.75, 0.25), 8)]
    for lo, hi, n in cases:
        verts, tris = W.box_mesh(lo, hi)
        g = np.arange(-n, 2 * n + 1) / n
        X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
        pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
        inside = np.all((pts > np.array(lo)) & (pts < np.array(hi)), axis=1)
        outside = np.any((pts < np.array(lo)) | (pts > np.array(hi)), axis=1)
        solid = orc.classify_points_3d(verts, tris, pts)
        assert inside.sum() > 0 and outside.sum() > 0
        np.testing.assert_array_equal(solid[inside], 1)
        np.testing.assert_array_equal(solid[outside], 0)
    verts, tris = W.box_mesh((0.25, 0.25, 0.25), (0.75, 0.75, 0.75))
    assert orc.classify_points_3d(verts, tris, np.array([[0.5, 0.5, 0.5]]))[0] == 1


def test_rotated_box_against_winding_number(orc):
    """A box turned about an oblique axis (no lattice alignment) and a lattice through its corners' region:
    classification equals the winding number at every node off the surface."""
    verts, tris = W.box_mesh((-0.3, -0.2, -0.25), (0.3, 0.2, 0.25))
    ax = np.array([1.0, 2.0, 3.0]) / np.sqrt(14.0)
    th = 0.7
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    Rm = np.eye(3) + np.sin(th) * K + (1 - np.cos(th)) * K @ K
    verts = verts @ Rm.T + 0.5
    g = (np.arange(24) + 0.5) / 24
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    wind = _winding(verts, tris, pts)
    keep = np.abs(wind - np.round(wind)) < 1e-6
    solid = orc.classify_points_3d(verts, tris, pts[keep])
    np.testing.assert_array_equal(solid, (wind[keep] > 0.5).astype(np.uint8))
    assert 100 < solid.sum() < keep.sum()
