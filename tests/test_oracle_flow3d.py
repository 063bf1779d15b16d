"""Pins of the 3-D oracle (oracle3d.c): the 3-D residual, stage update and halos against the pinned 2-D oracle,
the 3-D IB / ghost reconstruction against linear profiles at plane walls, and the 3-D force integral against
the divergence theorem.

The 2-D reduction: a 3-D field that does not vary along one axis (periodic there, no velocity along it) obeys
the 2-D equations in the other two, and the 3-D oracle adds every third-direction term to the 2-D oracle's
arithmetic in the same order, so its state must equal the 2-D oracle's bit for bit -- in each of the three
coordinate planes, which checks every face direction, every viscous cross term and every halo side of the
3-D code against the 2-D oracle (pinned by tests/test_oracle_flow.py).  A wrong index, a transposed derivative
or a dropped term in one direction breaks the equality in the planes that use it.
"""
import math

import numpy as np
import pytest

from paper_1912_11908_gb300 import workloads as W

FS, OUT, PER = W.BC_FREESTREAM, W.BC_OUTFLOW, W.BC_PERIODIC


def _field2d(nx, ny, lo, hi, uinf, mach, seed):
    """A smooth seeded perturbation of the free stream on a 2-D grid (conserved variables)."""
    rng = np.random.default_rng(seed)
    g = 1.4
    pinf = 1.0 / (g * mach * mach)
    x = lo[0] + (np.arange(nx) + 0.5) * (hi[0] - lo[0]) / nx
    y = lo[1] + (np.arange(ny) + 0.5) * (hi[1] - lo[1]) / ny
    X, Y = np.meshgrid(x, y)
    a = rng.uniform(0.5, 1.5, 8)
    ph = rng.uniform(0, 2 * np.pi, 8)
    r = 1.0 + 0.05 * np.sin(2 * np.pi * a[0] * X + ph[0]) * np.cos(2 * np.pi * a[1] * Y + ph[1])
    u = uinf[0] + 0.1 * np.sin(2 * np.pi * a[2] * Y + ph[2]) * np.cos(2 * np.pi * a[3] * X + ph[3])
    v = uinf[1] + 0.1 * np.cos(2 * np.pi * a[4] * X + ph[4]) * np.sin(2 * np.pi * a[5] * Y + ph[5])
    p = pinf * (1.0 + 0.05 * np.cos(2 * np.pi * a[6] * X + ph[6]) * np.sin(2 * np.pi * a[7] * Y + ph[7]))
    return np.stack([r, r * u, r * v, p / (g - 1.0) + 0.5 * r * (u * u + v * v)])


# the 2-D case: 20 x 16 cells, inflow / outflow in x, free stream in y, viscous, M 0.5
NX2, NY2, LO2, HI2, UINF2, BC2 = 20, 16, (0.0, -0.5), (1.25, 0.5), (0.8, 0.3), (FS, OUT, FS, FS)
MACH, RE, DT, NSTEPS, NINV = 0.5, 50.0, 2e-3, 4, 4


def _case_2d(orc):
    spec = W.case_spec(None, NX2, NY2, (LO2[0], HI2[0], LO2[1], HI2[1]), MACH, RE, BC2, uinf=UINF2, dt_fixed=DT)
    c = orc.Case(spec)
    c.set_state(_field2d(NX2, NY2, LO2, HI2, UINF2, MACH, 7))
    return c


def _embed(U2, plane):
    """3-D spec and state of the 2-D case laid in `plane`, constant along the remaining axis."""
    r, mu_, mv_, E = U2
    z = np.zeros_like(r)
    if plane == "xy":
        comps, n, axes = (r, mu_, mv_, z, E), (NX2, NY2, NINV), (0, 1)
    elif plane == "xz":
        comps, n, axes = (r, mu_, z, mv_, E), (NX2, NINV, NY2), (0, 2)
    else:
        comps, n, axes = (r, z, mu_, mv_, E), (NINV, NX2, NY2), (1, 2)
    inv = 3 - sum(axes)
    lo, hi, uinf, bc = [0.0] * 3, [1.0] * 3, [0.0] * 3, [PER] * 6
    for k2, a in enumerate(axes):
        lo[a], hi[a], uinf[a] = LO2[k2], HI2[k2], UINF2[k2]
        bc[2 * a], bc[2 * a + 1] = BC2[2 * k2], BC2[2 * k2 + 1]
    spec = W.case3d_spec(None, None, n, lo, hi, MACH, RE, bc, uinf=uinf, dt_fixed=DT)
    U3 = np.empty((5, n[2], n[1], n[0]))
    for v in range(5):
        c2 = comps[v]  # [y2][x2]
        if plane == "xy":
            U3[v] = np.broadcast_to(c2[None, :, :], U3[v].shape)
        elif plane == "xz":
            U3[v] = np.broadcast_to(c2[:, None, :], U3[v].shape)
        else:
            U3[v] = np.broadcast_to(c2[:, :, None], U3[v].shape)
    return spec, U3, inv


def _slices(U3, plane):
    """The 2-D-shaped slices of a 3-D state along its invariant axis, in the 2-D variable order."""
    idx = {"xy": (0, 1, 2, 4), "xz": (0, 1, 3, 4), "yz": (0, 2, 3, 4)}[plane]
    n_inv = {"xy": U3.shape[1], "xz": U3.shape[2], "yz": U3.shape[3]}[plane]
    for s in range(n_inv):
        if plane == "xy":
            yield U3[list(idx), s, :, :]
        elif plane == "xz":
            yield U3[list(idx), :, s, :]
        else:
            yield U3[list(idx), :, :, s]


@pytest.mark.parametrize("plane", ["xy", "xz", "yz"])
def test_3d_reduces_to_2d_bit_for_bit(orc, plane):
    c2 = _case_2d(orc)
    U0 = c2.state()
    c2.step(NSTEPS)
    ref = c2.state()
    spec, U3, inv = _embed(U0, plane)
    c3 = orc.Case3D(spec)
    c3.set_state(U3)
    c3.step(NSTEPS)
    out = c3.state()
    assert np.abs(ref - U0).max() > 1e-4  # the 2-D flow did evolve
    other = {"xy": 3, "xz": 2, "yz": 1}[plane]
    assert (out[other] == 0.0).all()  # no velocity appears along the invariant axis
    for s in _slices(out, plane):
        np.testing.assert_array_equal(s, ref)


def test_3d_free_stream_is_preserved(orc):
    """A uniform state in a periodic box stays uniform to round-off (the stage weights 3/4 + 1/4 and
    1/3 + 2/3 are not exact in binary)."""
    spec = W.case3d_spec(None, None, (8, 6, 5), (0, 0, 0), (1, 1, 1), 0.4, 100.0, (PER,) * 6,
                         uinf=(0.6, -0.3, 0.2), dt_fixed=1e-3)
    c = orc.Case3D(spec)
    U0 = c.state()
    c.step(3)
    np.testing.assert_allclose(c.state(), U0, rtol=2e-15, atol=1e-15)


def _sphere_case(orc, n=24, uinf=(0.0, 0.0, 0.0), mach=0.3, **kw):
    verts, tris = W.uv_sphere(radius=0.5)
    spec = W.case3d_spec(verts, tris, (n, n, n), (-1, -1, -1), (1, 1, 1), mach, 100.0, (FS,) * 6, uinf=uinf,
                         ref_area=math.pi * 0.25, **kw)
    return spec, orc.Case3D(spec)


def test_quiescent_sphere_stays_at_rest(orc):
    """Fluid at rest around a static body: IB and ghost reconstruction and the residual keep it at rest and
    uniform (Eq. 4-8 with a uniform state; any wrong sign or dropped weight would set it moving)."""
    spec, c = _sphere_case(orc, dt_fixed=1e-3)
    assert c.classify() == 0
    c.step(3)
    U = c.state()
    tags = c.tags()
    live = tags != 1  # every node the solver writes
    pinf = 1.0 / (1.4 * 0.09)
    assert np.abs(U[1:4][:, live]).max() < 1e-12
    p = 0.4 * (U[4] - 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0])
    assert np.abs(p[live] / pinf - 1.0).max() < 1e-13
    assert np.abs(U[0][live] - 1.0).max() < 1e-13


def test_stencil_geometry_invariants(orc):
    """Sec. 4.3 / Sec. 5 readings: the node lies on the line P' + xi n; an IB probe one cell diagonal beyond
    it, a ghost image point at its mirror position, each pushed out by min spacing per step; weights sum to 1
    and vanish on invalid corners; normals are unit vectors out of the body (the sphere's centre is behind)."""
    spec, c = _sphere_case(orc)
    assert c.classify() == 0
    st = c.stencils()
    n = spec["n"][0]
    d = 2.0 / n
    h = math.sqrt(3.0) * d
    node = st["node"]
    X = np.stack([-1 + (node % n + 0.5) * d, -1 + ((node // n) % n + 0.5) * d, -1 + (node // (n * n) + 0.5) * d], 1)
    np.testing.assert_allclose(st["b"] + st["xi_node"][:, None] * st["n"], X, rtol=0, atol=1e-14)
    ib = st["kind"] == 0
    np.testing.assert_allclose(st["xi_probe"][ib], st["xi_node"][ib] + h + st["nstep"][ib] * d, rtol=0, atol=1e-14)
    gh = ~ib
    mirror = np.maximum(-st["xi_node"][gh], 0.5 * d)
    np.testing.assert_allclose(st["xi_probe"][gh], mirror + st["nstep"][gh] * d, rtol=0, atol=1e-14)
    assert (st["xi_node"][ib] > 0).all() and (st["xi_node"][gh] < 0).all()
    assert (st["mask"] != 0).all()
    np.testing.assert_allclose(st["w"].sum(1), 1.0, rtol=0, atol=1e-14)
    bits = (st["mask"][:, None] >> np.arange(8)) & 1
    assert (st["w"][bits == 0] == 0).all()
    np.testing.assert_allclose(np.linalg.norm(st["n"], axis=1), 1.0, rtol=0, atol=1e-14)
    assert ((st["b"] * st["n"]).sum(1) > 0.45).all()  # P'.n > 0: n points away from the centre
    assert (st["mask"] == 255).mean() > 0.7
    assert set(np.unique(st["kind"])) == {0, 1, 2, 3}


def _rotation_to(nv):
    """A rotation matrix taking e_x to the unit vector nv."""
    nv = np.asarray(nv, float)
    a = np.array([0.0, 0.0, 1.0]) if abs(nv[2]) < 0.9 else np.array([1.0, 0.0, 0.0])
    t1 = np.cross(nv, a)
    t1 /= np.linalg.norm(t1)
    t2 = np.cross(nv, t1)
    return np.stack([nv, t1, t2], 1)


@pytest.mark.parametrize("oblique", [False, True])
def test_plane_wall_reproduces_linear_profiles(orc, oblique):
    """Eq. 4 / Sec. 5 at a plane wall: velocity linear in the distance s from the wall (zero on it), pressure
    and temperature uniform.  The IB value u_P xi_node / xi_probe and the ghost value through the mirror image
    point reproduce u = a s exactly wherever the cube is complete (trilinear is exact for linear fields) -- a
    wrong sign of the normal, a wrong image point or a dropped ratio fails it at every layer."""
    N = 24
    d = 1.0 / N
    if oblique:
        nrm = np.array([2.0, 2.0, 1.0]) / 3.0
        C0 = np.array([0.47, 0.52, 0.49])
    else:
        nrm = np.array([1.0, 0.0, 0.0])
        C0 = np.array([10 * d, 0.5, 0.5])  # the wall between cell planes 9 and 10
    verts, tris = W.box_mesh((-4.0, -4.0, -4.0), (0.0, 4.0, 4.0))  # its +x face is the wall
    verts = verts @ _rotation_to(nrm).T + C0
    spec = W.case3d_spec(verts, tris, (N, N, N), (0, 0, 0), (1, 1, 1), 0.3, 100.0, (FS,) * 6, uinf=(0, 0, 0))
    c = orc.Case3D(spec)
    nerr = c.classify()
    st = c.stencils()
    bad = st["node"][st["mask"] == 0]
    assert nerr == bad.size and (oblique or nerr == 0)
    # probes that leave the domain find no corner: only near the domain's sides, where the oblique wall meets them
    bi, bj, bk = bad % N, (bad // N) % N, bad // (N * N)
    assert (np.minimum.reduce([bi, bj, bk, N - 1 - bi, N - 1 - bj, N - 1 - bk]) < 3).all()
    xc = (np.arange(N) + 0.5) * d
    Z, Y, X = np.meshgrid(xc, xc, xc, indexing="ij")
    s = (X - C0[0]) * nrm[0] + (Y - C0[1]) * nrm[1] + (Z - C0[2]) * nrm[2]
    vel = np.array([0.7, -0.4, 0.25])
    g = 1.4
    pinf = 1.0 / (g * 0.09)
    r = np.ones_like(s)
    u, v, w = vel[0] * s, vel[1] * s, vel[2] * s
    c.set_state(np.stack([r, r * u, r * v, r * w, pinf / (g - 1.0) + 0.5 * r * (u * u + v * v + w * w)]))
    c.reconstruct()
    U = c.state()
    # complete cubes on the wall face, away from the domain's sides (where IB probes leave the domain and take
    # inverse-distance weights, and the image points that use those IB nodes inherit it)
    nd = st["node"]
    edge = np.minimum.reduce([nd % N, (nd // N) % N, nd // (N * N), N - 1 - nd % N, N - 1 - (nd // N) % N,
                              N - 1 - nd // (N * N)])
    ok = (st["mask"] == 255) & (np.abs(st["n"] @ nrm - 1.0) < 1e-12) & (edge >= 5)
    assert ok.mean() > 0.2
    # on the oblique wall every G1 image point (within one spacing of the wall) has a cube that straddles the
    # wall and takes inverse-distance weights; the axis-aligned wall puts them on the IB plane
    for kind in ((0, 2, 3) if oblique else range(4)):
        assert (ok & (st["kind"] == kind)).sum() >= 100, kind
    node = st["node"][ok]
    k, j, i = node // (N * N), (node // N) % N, node % N
    sn = s[k, j, i]
    for a in range(3):
        np.testing.assert_allclose(U[1 + a][k, j, i] / U[0][k, j, i], vel[a] * sn, rtol=0, atol=1e-13)
    p = (g - 1.0) * (U[4] - 0.5 * (U[1] ** 2 + U[2] ** 2 + U[3] ** 2) / U[0])
    np.testing.assert_allclose(p[k, j, i], pinf, rtol=1e-14)
    np.testing.assert_allclose(U[0][k, j, i], 1.0, rtol=1e-14)


def test_forces_of_linear_fields_on_a_box(orc):
    """Eq. 9 on a closed box (two triangles per face) with its faces midway between lattice planes: each
    triangle's probe, one cell diagonal out along the face normal from the centroid, has a cube of fluid nodes
    only, so any linear field is interpolated exactly and the force is the per-triangle sum of the integrand at
    the probes, evaluated here in closed form: pressure p_inf + G.x and velocity u = M x + u0 give
        F = sum_f [-(G.P_f) n_f + mu (u(P_f) - (u(P_f).n_f) n_f) / h] A_f,   P_f = m_f + h n_f
    -- a wrong normal, area, centroid, probe distance or tangential projection fails it."""
    N = 24
    d = 2.0 / N
    h = math.sqrt(3.0) * d
    verts, tris = W.box_mesh((-0.5, -0.5, -0.5), (0.5, 0.5, 0.5))
    spec = W.case3d_spec(verts, tris, (N, N, N), (-1, -1, -1), (1, 1, 1), 0.3, 100.0, (FS,) * 6, ref_area=2.0)
    c = orc.Case3D(spec)
    assert c.classify() == 0
    g = 1.4
    pinf = 1.0 / (g * 0.09)
    G = pinf * np.array([0.3, -0.2, 0.1])
    M = np.array([[0.1, 0.4, -0.2], [0.3, -0.1, 0.5], [-0.6, 0.2, 0.05]])
    u0 = np.array([0.2, -0.1, 0.3])
    xc = -1 + (np.arange(N) + 0.5) * d
    Z, Y, X = np.meshgrid(xc, xc, xc, indexing="ij")
    XYZ = np.stack([X, Y, Z])
    p = pinf + np.tensordot(G, XYZ, 1)
    vel = np.tensordot(M, XYZ, 1) + u0[:, None, None, None]
    r = p / pinf  # T = 1
    c.set_state(np.concatenate([r[None], r * vel, (p / (g - 1.0) + 0.5 * r * (vel ** 2).sum(0))[None]]))
    F = c.forces()
    mu = 1.0 / 100.0
    A, B, Cv = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    cr = np.cross(B - A, Cv - A)
    area = 0.5 * np.linalg.norm(cr, axis=1)
    nf = cr / np.linalg.norm(cr, axis=1)[:, None]
    P = (A + B + Cv) / 3.0 + h * nf
    uP = P @ M.T + u0
    ut = uP - (uP * nf).sum(1)[:, None] * nf
    expect = ((-(P @ G)[:, None] * nf + mu * ut / h) * area[:, None]).sum(0)
    np.testing.assert_allclose(F[3:], expect, rtol=0, atol=1e-12 * pinf)
    np.testing.assert_allclose(F[:3], F[3:] / (0.5 * 2.0), rtol=1e-15)
    assert np.abs(expect).min() > 1e-3


def test_forces_vanish_in_uniform_pressure(orc):
    """Eq. 9 on the 1200-triangle sphere at rest in a uniform pressure other than p_inf: the closed surface's
    sum of n A vanishes, whatever weights each probe takes."""
    spec, c = _sphere_case(orc)
    assert c.classify() == 0
    g, pinf = 1.4, 1.0 / (1.4 * 0.09)
    n = spec["n"][0]
    one = np.ones((n, n, n))
    c.set_state(np.stack([1.3 * one, 0 * one, 0 * one, 0 * one, 1.3 * pinf / (g - 1.0) * one]))
    F = c.forces()
    assert np.abs(F[3:]).max() < 1e-12 * pinf


def test_cfl_rule_in_closed_form(orc):
    """The CFL rule of the 3-D oracle on a uniform state (periodic box, so the state stays uniform):
    dt = CFL / ((|u|+c)/dx + (|v|+c)/dy + (|w|+c)/dz + 2 gamma mu / (Pr rho) (1/dx^2 + 1/dy^2 + 1/dz^2)), the rule
    written out here from the formula with c = sqrt(gamma p / rho) = 1 / M (free stream: rho = T = 1)."""
    n, lo, hi, mach, re, cfl, uinf = (10, 7, 6), (0.0, -1.0, 0.5), (2.0, 0.4, 1.7), 0.4, 80.0, 0.45, (0.7, -0.5, 0.3)
    spec = W.case3d_spec(None, None, n, lo, hi, mach, re, (PER,) * 6, uinf=uinf, cfl=cfl)
    c = orc.Case3D(spec)
    c.step(1)
    d = [(hi[a] - lo[a]) / n[a] for a in range(3)]
    cs = 1.0 / mach
    lam = sum((abs(uinf[a]) + cs) / d[a] for a in range(3)) + \
        (2.0 * 1.4 * (1.0 / re) / 0.72) * sum(1.0 / (d[a] * d[a]) for a in range(3))
    assert abs(c.last_dt() - cfl / lam) <= 1e-14 * (cfl / lam)
    assert abs(c.time() - cfl / lam) <= 1e-14 * (cfl / lam)
