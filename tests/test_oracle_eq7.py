"""Pins of the oracle's supersonic moving-body pressure condition (Eq. 7).

For a body moving faster than the free-stream sound speed, the wall pressure
gradient along the normal carries the centripetal term of the normal momentum
balance, rho u_t^2 kappa, on top of the body-acceleration term of Eq. 6.
The pins check the two ingredients against what geometry and the Euler
equations fix: the local curvature against circles and a smooth non-convex
curve in closed form, and the IB-node pressure against an exact steady Euler
solution with curved streamlines (a swirling flow around a translating
cylinder), where the condition must remove the first-order pressure error
that the plain acceleration condition leaves.
"""
import math

import numpy as np

from paper_1912_11908_gb300 import workloads as W


def _all_stencils(c):
    return np.concatenate([c.stencils(k) for k in range(4)])


def test_curvature_on_regular_polygons_is_inverse_radius(orc):
    """Three vertices of a regular polygon lie on its circumscribed circle, so the vertex curvature, and any
    interpolation between equal vertex values, is exactly 1/r (positive: the counter-clockwise body turns
    left at every vertex).  The tolerance is the rounding of the vertex coordinates, amplified by the cross
    product of nearly parallel edges (about eps / (edge * turning angle))."""
    for n, d, grid in ((256, 1.0, 96), (64, 2.4, 80), (1000, 0.6, 120)):
        verts = W.cylinder(n, d, center=(0.1, -0.05))
        spec = W.case_spec(verts, grid, grid, (-1.5, 1.5, -1.5, 1.5), 0.5, 100.0, W.FAR)
        c = orc.Case(spec)
        assert c.classify() == 0
        s = _all_stencils(c)
        assert len(s) > 50
        np.testing.assert_allclose(s["curv"], 2.0 / d, rtol=1e-9, atol=0)


def test_curvature_of_smooth_nonconvex_curve(orc):
    """r(theta) = 1 + a cos(3 theta) has convex lobes and concave waists.  The signed curvature
    (r^2 + 2 r'^2 - r r'') / (r^2 + r'^2)^(3/2) of the curve at the boundary point's polar angle matches the
    stencil's to the discretisation error, including the sign change in the waists."""
    a, n = 0.25, 3000
    th = 2.0 * math.pi * np.arange(n) / n
    r = 1.0 + a * np.cos(3 * th)
    verts = np.stack([r * np.cos(th), r * np.sin(th)], 1)
    spec = W.case_spec(verts, 200, 200, (-1.5, 1.5, -1.5, 1.5), 0.5, 100.0, W.FAR)
    c = orc.Case(spec)
    assert c.classify() == 0
    s = _all_stencils(c)
    t = np.arctan2(s["by"], s["bx"])
    rr = 1.0 + a * np.cos(3 * t)
    r1 = -3 * a * np.sin(3 * t)
    r2 = -9 * a * np.cos(3 * t)
    kappa = (rr * rr + 2 * r1 * r1 - rr * r2) / (rr * rr + r1 * r1) ** 1.5
    assert kappa.min() < -2.0 and kappa.max() > 2.0  # both signs are exercised
    assert np.abs(s["curv"] - kappa).max() < 2e-3


def _swirl_state(spec, V, Wt, p0, rho0=1.0, rmin=0.3, r0=0.5):
    """Lab-frame field of a cylinder of radius r0 centred at the origin moving at V: in the body frame a
    steady swirl u_theta = Wt at constant density, an exact steady Euler solution whose radial balance
    dp/dr = rho u_theta^2 / r gives p = p0 + rho Wt^2 ln(r / r0) (clipped inside the body)."""
    nx, ny = spec["nx"], spec["ny"]
    x0, x1, y0, y1 = spec["domain"]
    X, Y = np.meshgrid(x0 + (np.arange(nx) + 0.5) * (x1 - x0) / nx, y0 + (np.arange(ny) + 0.5) * (y1 - y0) / ny)
    R = np.maximum(np.hypot(X, Y), 1e-12)
    u = V[0] - Wt * Y / R
    v = V[1] + Wt * X / R
    p = p0 + rho0 * Wt * Wt * np.log(np.maximum(R, rmin) / r0)
    r = np.full_like(X, rho0)
    g = spec["gamma"]
    return np.stack([r, r * u, r * v, p / (g - 1.0) + 0.5 * r * (u * u + v * v)]), p, X, Y


def _ib_pressure_errors(orc, uinf, V, Wt=0.6):
    spec = W.case_spec(W.cylinder(256, 1.0), 128, 128, (-1.0, 1.0, -1.0, 1.0), 2.0, 100.0, W.FAR,
                       uinf=uinf, motion=W.MOTION_CONST, vel=V)
    c = orc.Case(spec)
    assert c.classify() == 0
    g = spec["gamma"]
    p0 = 1.0 / (g * spec["mach"] ** 2)
    U, p_exact, X, Y = _swirl_state(spec, V, Wt, p0)
    c.set_state(U)
    c.reconstruct(0.0)
    U2 = c.state()
    nx = spec["nx"]
    err = []
    for s in c.stencils(0):
        if s["mask"] != 15:
            continue
        i, j = s["cell"] % nx, s["cell"] // nx
        r, mx, my, E = U2[:, j, i]
        p = (g - 1.0) * (E - 0.5 * (mx * mx + my * my) / r)
        err.append(p - p_exact[j, i])
    assert len(err) > 100
    return np.array(err)


def test_eq7_recovers_the_radial_balance_of_a_swirling_flow(orc):
    """Body at speed 1 in gas at rest, sound speed 1/2: Eq. 7 applies, and the IB-node pressure matches the
    exact p(r) to second order in the node-probe distance.  The same field with the body moving with the
    free stream (relative speed 0, Eq. 7 off) keeps the first-order error rho Wt^2 (xi_p - xi_n) / r0 of the
    plain condition, whose sign (node pressure too high) the added term must cancel, not double."""
    e_on = _ib_pressure_errors(orc, uinf=(0.0, 0.0), V=(1.0, 0.0))
    e_off = _ib_pressure_errors(orc, uinf=(1.0, 0.0), V=(1.0, 0.0))
    assert e_off.min() > 0.0  # without the term the extrapolated node pressure overshoots everywhere
    assert np.abs(e_on).max() < 0.15 * np.abs(e_off).max()
    assert np.abs(e_on).mean() < 0.1 * np.abs(e_off).mean()


def test_eq7_applies_only_above_the_free_stream_sound_speed(orc):
    """The criterion compares the body's speed relative to the free stream with c_inf = 1/M: at 0.9 c_inf
    the node pressure is the plain condition's (bit-identical to the body moving with the stream), at
    1.1 c_inf it is corrected."""
    c_inf = 0.5
    e_ref = _ib_pressure_errors(orc, uinf=(0.9 * c_inf, 0.0), V=(0.9 * c_inf, 0.0))
    e_sub = _ib_pressure_errors(orc, uinf=(0.0, 0.0), V=(0.9 * c_inf, 0.0))
    e_sup = _ib_pressure_errors(orc, uinf=(0.0, 0.0), V=(1.1 * c_inf, 0.0))
    assert np.array_equal(e_sub, e_ref)
    assert np.abs(e_sup).max() < 0.15 * np.abs(e_sub).max()


def test_supersonic_body_translating_with_stream_is_preserved(orc):
    """M = 2 stream with the body moving at the stream velocity: no velocity relative to the wall, so the
    added term vanishes and the uniform field stays uniform over re-classified steps."""
    spec = W.case_spec(W.cylinder(64, 1.0), 96, 48, (-2.0, 6.0, -2.0, 2.0), 2.0, 100.0, W.SUPERSONIC,
                       motion=W.MOTION_CONST, vel=(1.0, 0.0))
    c = orc.Case(spec)
    U0 = c.state()
    c.step(40)
    assert c.time() > 0.2
    U1 = c.state()
    live = c.tags() != 1
    for k in range(4):
        assert np.abs(U1[k] - U0[k])[live].max() <= 1e-12 * max(1.0, np.abs(U0[k]).max()), k


def test_wall_pressure_stays_positive_under_a_strong_centripetal_gradient(orc):
    """With T fixed along the normal (Eq. 8), dp/dn = rho G = p G / (R T) integrates to an exponential, so the
    rebuilt pressure stays positive however large the gradient is against the grid spacing.  Swirl W = 2 at
    M = 2 on a 64 x 64 grid: the ghost layers sit where rho W^2 kappa times the extrapolation distance exceeds
    the wall pressure (a linear extrapolation would go negative); every rebuilt node keeps p > 0."""
    spec = W.case_spec(W.cylinder(256, 1.0), 64, 64, (-1.0, 1.0, -1.0, 1.0), 2.0, 100.0, W.FAR,
                       uinf=(0.0, 0.0), motion=W.MOTION_CONST, vel=(1.0, 0.0))
    c = orc.Case(spec)
    assert c.classify() == 0
    g = spec["gamma"]
    p0 = 1.0 / (g * spec["mach"] ** 2)
    U, _, _, _ = _swirl_state(spec, (1.0, 0.0), 2.0, p0, rmin=0.5)
    c.set_state(U)
    c.reconstruct(0.0)
    U2 = c.state()
    nx = spec["nx"]
    ps, ratio = [], []
    for kind in range(4):
        for s in c.stencils(kind):
            i, j = s["cell"] % nx, s["cell"] // nx
            r, mx, my, E = U2[:, j, i]
            p = (g - 1.0) * (E - 0.5 * (mx * mx + my * my) / r)
            # the field's pressure at the probe / image point, in closed form
            rp = math.hypot(s["bx"] + s["xi_probe"] * s["nx"], s["by"] + s["xi_probe"] * s["ny"])
            ps.append(p)
            ratio.append(p / (p0 + 4.0 * math.log(max(rp, 0.5) / 0.5)))
    ps = np.array(ps)
    assert np.isfinite(ps).all() and ps.min() > 0.0
    # node / probe pressure below exp(-1.2): the linear form 1 - x, x > 1.2, would be negative there
    assert min(ratio) < 0.3
