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
