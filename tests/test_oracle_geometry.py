"""Pins of the FP64 oracle's geometry against brute force, exact arithmetic and closed forms.

Sec. 3.2 (ray-casting classification, IB / ghost tagging), Sec. 4.1 (closest
feature), Sec. 4.2 (pseudo-normals), Sec. 4.3-4.6 and Sec. 5 (boundary point,
probe / image point, interpolation stencil), Sec. 6 (force integral).
"""
import math
from fractions import Fraction

import numpy as np

from paper_1912_11908_gb300 import workloads as W

FLUID, SOLID, IB, G1, G2, G3 = range(6)


def _exact_inside(verts, px, py):
    """Exact-rational ray parity with the same half-open crossing convention."""
    P = (Fraction(px), Fraction(py))
    odd = False
    n = len(verts)
    for k in range(n):
        ax, ay = (Fraction(v) for v in verts[k])
        bx, by = (Fraction(v) for v in verts[(k + 1) % n])
        if (ay > P[1]) != (by > P[1]):
            xint = ax + (P[1] - ay) * (bx - ax) / (by - ay)
            if xint > P[0]:
                odd = not odd
    return odd


def _dist_to_polyline(verts, px, py):
    best = math.inf
    n = len(verts)
    for k in range(n):
        a = np.array(verts[k])
        b = np.array(verts[(k + 1) % n])
        e = b - a
        t = np.clip(np.dot([px, py] - a, e) / np.dot(e, e), 0.0, 1.0)
        best = min(best, float(np.hypot(*(a + t * e - [px, py]))))
    return best


def test_ray_parity_matches_exact_arithmetic(orc):
    rng = np.random.default_rng(11)
    disagreements = 0
    for trial in range(12):
        verts = W.random_polygon(rng, int(rng.integers(3, 24)), rmin=0.2, rmax=1.0)
        # put some vertices exactly on grid-line ordinates to exercise the half-open rule
        grid = (np.arange(24) + 0.5) / 12.0 - 1.0
        for k in range(0, len(verts), 3):
            verts[k, 1] = grid[int(rng.integers(0, 24))]
        X, Y = np.meshgrid(grid, grid)
        pts = np.stack([X.ravel(), Y.ravel()], axis=1)
        got = orc.classify_points(verts, pts)
        for n, (px, py) in enumerate(pts):
            ex = _exact_inside(verts.tolist(), px, py)
            if bool(got[n]) != ex:
                # only acceptable within rounding of the surface
                assert _dist_to_polyline(verts, px, py) < 1e-12
                disagreements += 1
    assert disagreements == 0


def test_ray_parity_cylinder_matches_disk(orc):
    verts = W.cylinder(256, 1.0)
    rng = np.random.default_rng(4)
    pts = rng.uniform(-0.7, 0.7, (4000, 2))
    r = np.hypot(pts[:, 0], pts[:, 1])
    keep = np.abs(r - 0.5) > 1e-4  # away from the 256-gon / circle difference (max 3.8e-5)
    got = orc.classify_points(verts, pts[keep])
    np.testing.assert_array_equal(got.astype(bool), r[keep] < 0.5)


def _tags_by_definition(solid):
    ny, nx = solid.shape
    tags = np.where(solid, SOLID, FLUID).astype(np.uint8)
    for j in range(ny):
        for i in range(nx):
            nb = [(i + di, j + dj) for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1))]
            if not solid[j, i]:
                if any(0 <= a < nx and 0 <= b < ny and solid[b, a] for a, b in nb):
                    tags[j, i] = IB
            else:
                for k in (1, 2, 3):
                    if any(0 <= i + k * di < nx and 0 <= j + k * dj < ny and not solid[j + k * dj, i + k * di]
                           for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1))):
                        tags[j, i] = G1 + k - 1
                        break
    return tags


def test_tags_and_lists_by_definition(orc):
    rng = np.random.default_rng(7)
    for trial in range(6):
        verts = W.random_polygon(rng, 9, rmin=0.3, rmax=0.9)
        spec = W.case_spec(verts, 30, 26, (-1.1, 1.1, -1.0, 1.0), 0.5, 100.0, W.FAR)
        c = orc.Case(spec)
        c.classify()
        tags = c.tags()
        xc = -1.1 + (np.arange(30) + 0.5) * 2.2 / 30
        yc = -1.0 + (np.arange(26) + 0.5) * 2.0 / 26
        X, Y = np.meshgrid(xc, yc)
        solid = orc.classify_points(verts, np.stack([X.ravel(), Y.ravel()], 1)).reshape(26, 30).astype(bool)
        np.testing.assert_array_equal(tags, _tags_by_definition(solid))
        for kind, tag in ((0, IB), (1, G1), (2, G2), (3, G3)):
            st = c.stencils(kind)
            np.testing.assert_array_equal(st["cell"], np.flatnonzero(tags.ravel() == tag))


def test_vertex_pseudo_normals_radial_on_regular_polygon(orc):
    verts = W.cylinder(256, 1.0)
    spec = W.case_spec(verts, 8, 8, (-1, 1, -1, 1), 0.5, 100.0, W.FAR)
    c = orc.Case(spec)
    n = c.vertex_normals()
    radial = verts / np.linalg.norm(verts, axis=1, keepdims=True)
    np.testing.assert_allclose(n, radial, atol=1e-14)


def test_pseudo_normal_sign_matches_parity_near_sharp_edges(orc):
    """Angle-weighted pseudo-normals classify points correctly by the sign of (X - C).n at every
    feature, including the sharp trailing edge (the property that motivates Sec. 4.2)."""
    verts = W.naca00xx(0.12, 100, 10.0)
    spec = W.case_spec(verts, 8, 8, (-1, 2, -1, 1), 0.5, 100.0, W.FAR)
    c = orc.Case(spec)
    vn = c.vertex_normals()
    e = np.roll(verts, -1, axis=0) - verts
    sn = np.stack([e[:, 1], -e[:, 0]], 1) / np.linalg.norm(e, axis=1, keepdims=True)
    rng = np.random.default_rng(9)
    te = verts[0]
    pts = np.concatenate([te + rng.normal(scale=0.01, size=(1500, 2)),
                          verts[rng.integers(0, len(verts), 1500)] + rng.normal(scale=0.01, size=(1500, 2))])
    inside = orc.classify_points(verts, pts).astype(bool)
    checked = 0
    for (px, py), ins in zip(pts, inside):
        f, region, cx, cy, d2 = c.closest(px, py)
        if d2 < 1e-20:
            continue
        n = sn[f] if region == 0 else vn[f]
        s = (px - cx) * n[0] + (py - cy) * n[1]
        assert (s < 0) == ins, (px, py, region, f)
        checked += 1
    assert checked > 2900


def test_closest_feature_against_dense_sampling(orc):
    verts = W.naca00xx(0.12, 60, 5.0)
    spec = W.case_spec(verts, 8, 8, (-1, 2, -1, 1), 0.5, 100.0, W.FAR)
    c = orc.Case(spec)
    rng = np.random.default_rng(3)
    t = np.linspace(0.0, 1.0, 2001)
    samples = np.concatenate([verts[k] + t[:, None] * (verts[(k + 1) % len(verts)] - verts[k])
                              for k in range(len(verts))])
    for _ in range(200):
        px, py = rng.uniform([-0.2, -0.3], [1.2, 0.3])
        f, region, cx, cy, d2 = c.closest(px, py)
        dmin = np.min(np.hypot(samples[:, 0] - px, samples[:, 1] - py))
        assert math.sqrt(d2) <= dmin + 1e-12
        assert math.sqrt(d2) >= dmin - 1e-3 * 0.05  # sampling resolution
        assert _dist_to_polyline(verts, cx, cy) < 1e-12


def test_stencil_geometry(orc):
    """Boundary point on the surface, node on the line through it along the local normal, probe or
    image point where the stencil says, weights a partition of unity over valid corners."""
    for spec in (W.cylinder_m02_re40(), W.wedge_m2_re1e4(192, 96),
                 W.case_spec(W.naca00xx(0.12, 400, 5.0), 256, 128, (-0.5, 1.5, -0.5, 0.5), 0.5, 1000.0, W.FAR)):
        c = orc.Case(spec)
        assert c.classify() == 0
        tags = c.tags()
        nx, ny = spec["nx"], spec["ny"]
        x0, x1, y0, y1 = spec["domain"]
        dx, dy = (x1 - x0) / nx, (y1 - y0) / ny
        verts = spec["verts"]
        for kind in range(4):
            for s in c.stencils(kind):
                i, j = s["cell"] % nx, s["cell"] // nx
                px, py = x0 + (i + 0.5) * dx, y0 + (j + 0.5) * dy
                assert _dist_to_polyline(verts, s["bx"], s["by"]) < 1e-12
                if s["region"] != 2:
                    cross = (px - s["bx"]) * s["ny"] - (py - s["by"]) * s["nx"]
                    assert abs(cross) < 1e-12
                    assert abs((px - s["bx"]) * s["nx"] + (py - s["by"]) * s["ny"] - s["xi_node"]) < 1e-12
                assert (s["xi_node"] >= 0) == (kind == 0) or s["xi_node"] == 0
                assert s["mask"] != 0
                w = s["w"]
                assert abs(w.sum() - 1.0) < 1e-13 and (w >= -1e-15).all()
                allowed = {FLUID} if kind == 0 else {FLUID, IB}
                for k in range(4):
                    ci, cj = s["i0"] + (k & 1), s["j0"] + (k >> 1)
                    if w[k] != 0:
                        assert 0 <= ci < nx and 0 <= cj < ny and tags[cj, ci] in allowed
                X = s["bx"] + s["xi_probe"] * s["nx"]
                Y = s["by"] + s["xi_probe"] * s["ny"]
                assert x0 + (s["i0"] + 0.5) * dx <= X + 1e-12 <= x0 + (s["i0"] + 1.5) * dx + 2e-12
                assert y0 + (s["j0"] + 0.5) * dy <= Y + 1e-12 <= y0 + (s["j0"] + 1.5) * dy + 2e-12


def test_ib_velocity_exact_for_linear_wall_field(orc):
    """A velocity field that vanishes on a flat face and varies linearly is reproduced exactly at IB nodes
    whose boundary point lies on that face (Dirichlet Eq. 4, bilinear probe, linear profile)."""
    a = math.radians(30.0)
    sq = np.array([[-0.5, -0.5], [0.5, -0.5], [0.5, 0.5], [-0.5, 0.5]])
    verts = sq @ np.array([[math.cos(a), math.sin(a)], [-math.sin(a), math.cos(a)]])
    spec = W.case_spec(verts, 64, 64, (-1.0, 1.0, -1.0, 1.0), 0.5, 100.0, W.FAR, uinf=(0.0, 0.0))
    c = orc.Case(spec)
    c.classify()
    nx = ny = 64
    xc = -1.0 + (np.arange(nx) + 0.5) * 2.0 / nx
    X, Y = np.meshgrid(xc, xc)
    f = 2  # face from vertex 2 to 3
    e = verts[3] - verts[2]
    n = np.array([e[1], -e[0]]) / np.linalg.norm(e)
    dist = (X - verts[2][0]) * n[0] + (Y - verts[2][1]) * n[1]
    u = 0.3 * dist
    v = -0.2 * dist
    r = np.ones_like(X)
    p = np.full_like(X, 1.0 / (1.4 * 0.25))
    U = np.stack([r, r * u, r * v, p / 0.4 + 0.5 * r * (u * u + v * v)])
    c.set_state(U)
    c.reconstruct(0.0)
    U2 = c.state()
    checked = 0
    for s in c.stencils(0):
        on_face = abs((s["bx"] - verts[2][0]) * n[0] + (s["by"] - verts[2][1]) * n[1]) < 1e-12
        if not on_face or s["mask"] != 15 or s["region"] == 2:
            continue
        i, j = s["cell"] % nx, s["cell"] // nx
        assert abs(U2[1, j, i] / U2[0, j, i] - u[j, i]) < 1e-12
        assert abs(U2[2, j, i] / U2[0, j, i] - v[j, i]) < 1e-12
        checked += 1
    assert checked >= 10


def test_force_integral_uniform_and_linear_pressure(orc):
    """Eq. 9: zero force for uniform pressure; for p = p_inf + g y sampled one diagonal spacing out along
    each segment normal the midpoint rule gives F = -g (A + h sum n_y^2 L) in y and -g h sum n_x n_y L in x.
    Probes whose square holds an IB corner use inverse-distance weights, which reproduce a linear field
    only approximately, hence the 1% tolerance (a sign, normal or length error is off by O(1))."""
    verts = W.cylinder(64, 1.0)
    spec = W.case_spec(verts, 80, 80, (-2.0, 2.0, -2.0, 2.0), 0.5, 0.0, W.FAR, uinf=(0.0, 0.0))
    c = orc.Case(spec)
    c.classify()
    np.testing.assert_allclose(c.forces(), 0.0, atol=1e-12)
    nx = ny = 80
    xc = -2.0 + (np.arange(nx) + 0.5) * 4.0 / nx
    X, Y = np.meshgrid(xc, xc)
    pinf = 1.0 / (1.4 * 0.25)
    g = 0.37
    p = pinf + g * Y
    r = np.ones_like(X)
    c.set_state(np.stack([r, 0 * r, 0 * r, p / 0.4]))
    F = c.forces()
    e = np.roll(verts, -1, axis=0) - verts
    L = np.linalg.norm(e, axis=1)
    nrm = np.stack([e[:, 1], -e[:, 0]], 1) / L[:, None]
    area = 0.5 * np.sum(verts[:, 0] * np.roll(verts[:, 1], -1) - np.roll(verts[:, 0], -1) * verts[:, 1])
    h = math.hypot(4.0 / nx, 4.0 / ny)
    fy = -g * (area + h * np.sum(nrm[:, 1] ** 2 * L))
    fx = -g * h * np.sum(nrm[:, 0] * nrm[:, 1] * L)
    assert abs(F[2] - fx) < 1e-12
    assert abs(F[3] / fy - 1.0) < 1e-2, (F, fy)


def _shear_layer_case(orc, vel, gammas, re=50.0, segs_per_face=4):
    """Rectangle whose faces sit a quarter cell from the nearest outside node row (sides (n + 1/2) dx), so that
    every force probe one diagonal spacing out has four FLUID corners; outside each face, within the face's
    strip, the gas slides parallel to the face with u = V + gamma_k d t_k (d the distance from the face)."""
    n = 128
    d = 4.0 / n
    lo, hi = -2.0 + 47.75 * d, -2.0 + 80.25 * d  # nodes at lo - d/4 and hi + d/4 are the first outside rows
    corners = [(lo, lo), (hi, lo), (hi, hi), (lo, hi)]
    verts = []
    for k in range(4):
        a, b = np.array(corners[k]), np.array(corners[(k + 1) % 4])
        for s in range(segs_per_face):
            verts.append(a + (b - a) * s / segs_per_face)
    verts = np.array(verts)
    motion = dict(motion=W.MOTION_CONST, vel=vel) if any(vel) else {}
    spec = W.case_spec(verts, n, n, (-2.0, 2.0, -2.0, 2.0), 0.2, re, W.FAR, **motion)
    c = orc.Case(spec)
    xc = -2.0 + (np.arange(n) + 0.5) * d
    X, Y = np.meshgrid(xc, xc)
    u = np.full_like(X, vel[0])
    v = np.full_like(X, vel[1])
    tang = [(1.0, 0.0), (0.0, 1.0), (-1.0, 0.0), (0.0, -1.0)]  # CCW: bottom, right, top, left
    inx, iny = (X >= lo) & (X <= hi), (Y >= lo) & (Y <= hi)
    dist = [np.where(inx & (Y < lo), lo - Y, -1.0), np.where(iny & (X > hi), X - hi, -1.0),
            np.where(inx & (Y > hi), Y - hi, -1.0), np.where(iny & (X < lo), lo - X, -1.0)]
    for k in range(4):
        m = dist[k] > 0.0
        u[m] += gammas[k] * dist[k][m] * tang[k][0]
        v[m] += gammas[k] * dist[k][m] * tang[k][1]
    r = np.ones_like(X)
    pinf = 1.0 / (1.4 * 0.04)
    c.set_state(np.stack([r, r * u, r * v, pinf / 0.4 + 0.5 * r * (u * u + v * v)]))
    face_of_seg = np.repeat(np.arange(4), segs_per_face)
    L = (hi - lo) / segs_per_face
    mu = 1.0 / re
    F = mu * L * segs_per_face * sum(gammas[k] * np.array(tang[k]) for k in range(4))
    return c, face_of_seg, mu, F


def test_force_integral_wall_shear_closed_form(orc):
    """Eq. 9's viscous term: in a gas sliding along each face of a rectangle with u_t = gamma_k d (a linear
    shear layer, exact wall shear mu gamma_k), every segment's skin friction is 2 mu gamma_k / (rho U^2) and the
    net force is mu L sum_k gamma_k t_k: the traction acts along +t where the gas outruns the wall.  Shear rates
    of both signs and different sizes per face, a body at rest and one translating at constant velocity with
    the gas carried along (only the velocity relative to the wall shears), two Reynolds numbers.  A sign,
    factor, probe-distance or relative-velocity error in tau_w = mu (u_P - U_wall).t / h fails it."""
    for vel in ((0.0, 0.0), (0.3, -0.2)):
        for re, gammas in ((50.0, (1.0, -2.0, 0.5, -1.5)), (400.0, (-0.7, 0.3, 2.0, 1.1))):
            c, face, mu, F = _shear_layer_case(orc, vel, gammas, re)
            cp, cf = c.surface()
            assert np.all(np.isfinite(cf))
            np.testing.assert_allclose(cf, 2.0 * mu * np.array(gammas)[face], rtol=1e-12, atol=1e-14)
            np.testing.assert_allclose(cp, 0.0, atol=1e-9)
            f = c.forces()
            np.testing.assert_allclose(f[2:], F, rtol=1e-12, atol=1e-14)
            np.testing.assert_allclose(f[:2], F / 0.5, rtol=1e-12, atol=1e-14)
