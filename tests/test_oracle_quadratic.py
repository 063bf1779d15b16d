"""Pins of the oracle's quadratic IB / ghost reconstruction (Sec. 4.5 and Sec. 5, the incompressible form).

Reading: along the local normal, quadratics in the distance s from the boundary point P' through the wall
condition at s = 0 and two probes -- the first where the linear form puts it (one diagonal spacing beyond an IB
node, the mirror image point of a ghost node), the second one diagonal spacing beyond the first.  Velocity is
Dirichlet (Eq. 4), temperature adiabatic (Eq. 8, zero wall slope), pressure takes the wall slope rho G of Eq. 5-7.

The pin: on a wall at 45 degrees with square cells, moving one diagonal spacing along the normal moves by
exactly one cell in x and in y.  With the wall on a line of cell centres, every IB probe and every ghost image
point lands on a cell centre, where the bilinear / inverse-distance interpolation returns the cell's own value.
A field that is quadratic in s with the right wall conditions is then reproduced exactly by the quadratic form,
at IB nodes and at all three ghost layers, while the linear form is off by O(h^2) -- a dropped term, a wrong
Lagrange weight or a wrong sign in the extrapolation fails one of the two checks.  (The cells on the wall line
are fluid here, so the IB nodes sit at s = 0: the velocity there is the wall's in both forms, while temperature
and pressure come from the zero-slope quadratic through the probes at h and 2h, which the linear form replaces
by the first probe's value.)
"""
import math

import numpy as np
import pytest

from paper_1912_11908_gb300 import workloads as W

N = 64
C = (62 + 1) / N  # the wall x + y = C passes through the cell centres with i + j = 62


def _spec(interp):
    # the body is the half-plane x + y < C inside the domain: a large triangle with its hypotenuse on the wall
    verts = np.array([[-1.0, -1.0], [C + 1.0, -1.0], [-1.0, C + 1.0]])
    return W.case_spec(verts, N, N, (0.0, 1.0, 0.0, 1.0), 0.3, 100.0, W.FAR, uinf=(0.0, 0.0), ib_interp=interp)


def _field(spec):
    """Quadratic profiles in s = (x + y - C) / sqrt(2) meeting the wall conditions of a static wall."""
    g, mach = spec["gamma"], spec["mach"]
    R = 1.0 / (g * mach * mach)  # p_inf; T_inf = 1 with rho_inf = 1
    xc = (np.arange(N) + 0.5) / N
    X, Y = np.meshgrid(xc, xc)
    s = (X + Y - C) / math.sqrt(2.0)
    u = 0.7 * s - 3.1 * s * s
    v = -0.4 * s + 2.3 * s * s
    T = 1.0 + 5.0 * s * s
    p = R * (1.0 + 4.0 * s * s)
    r = p / (R * T)
    U = np.stack([r, r * u, r * v, p / (g - 1.0) + 0.5 * r * (u * u + v * v)])
    return U, s, (p, u, v, T), R


def _reconstructed_errors(orc, interp):
    spec = _spec(interp)
    c = orc.Case(spec)
    assert c.classify() == 0
    U, s, (p, u, v, T), R = _field(spec)
    c.set_state(U)
    c.reconstruct(0.0)
    U2 = c.state()
    g = spec["gamma"]
    out = {k: [] for k in range(4)}
    for kind in range(4):
        for st in c.stencils(kind):
            i, j = st["cell"] % N, st["cell"] // N
            # ghost nodes on the wall itself (s = 0: the image point is pushed off the mirror position) and
            # nodes near the domain sides, whose probes leave the domain, are not part of the pin
            if (kind > 0 and abs(s[j, i]) < 1e-9) or min(i, j) < 4 or max(i, j) > N - 12:
                continue
            r, mx, my, E = U2[:, j, i]
            uu, vv = mx / r, my / r
            pp = (g - 1.0) * (E - 0.5 * r * (uu * uu + vv * vv))
            TT = pp / (r * R)
            scale = np.array([R, 1.0, 1.0, 1.0])
            err = np.abs(np.array([pp - p[j, i], uu - u[j, i], vv - v[j, i], TT - T[j, i]])) / scale
            out[kind].append(err.max())
    return out, c


def test_quadratic_form_reproduces_quadratic_profiles_exactly(orc):
    out, c = _reconstructed_errors(orc, W.INTERP_QUADRATIC)
    for kind in range(4):
        assert len(out[kind]) >= 20, (kind, len(out[kind]))  # IB nodes and all three ghost layers checked
        assert max(out[kind]) < 1e-11, (kind, max(out[kind]))
    # the second probe sits one diagonal spacing beyond the first, on a cell centre
    h = math.sqrt(2.0) / N
    for kind in range(4):
        st = c.stencils(kind)
        ok = st["maskb"] != 0
        assert ok.mean() > 0.9
        np.testing.assert_allclose(st["xi_probe2"][ok] - st["xi_probe"][ok], h, rtol=0, atol=1e-12)


def test_linear_form_is_off_by_second_order(orc):
    """The same field through the compressible (linear) form: errors of order beta h^2 at every layer, so the
    pin above separates the two forms."""
    out, c = _reconstructed_errors(orc, W.INTERP_LINEAR)
    for kind in range(4):
        assert len(out[kind]) >= 20
        assert min(out[kind]) > 1e-5, (kind, min(out[kind]))
    assert (c.stencils(0)["maskb"] == 0).all()  # no second probe in the linear form


def test_quadratic_matches_linear_for_linear_profiles(orc):
    """Fields linear in s (with zero-slope temperature and pressure, i.e. uniform) are reproduced by both
    forms: the quadratic form reduces to the linear one when the profile has no curvature."""
    res = {}
    for interp in (W.INTERP_LINEAR, W.INTERP_QUADRATIC):
        spec = _spec(interp)
        c = orc.Case(spec)
        c.classify()
        g, R = spec["gamma"], 1.0 / (spec["gamma"] * spec["mach"] ** 2)
        xc = (np.arange(N) + 0.5) / N
        X, Y = np.meshgrid(xc, xc)
        s = (X + Y - C) / math.sqrt(2.0)
        u, v = 0.5 * s, -0.25 * s
        r = np.ones_like(s)
        p = np.full_like(s, R)
        c.set_state(np.stack([r, r * u, r * v, p / (g - 1.0) + 0.5 * r * (u * u + v * v)]))
        c.reconstruct(0.0)
        res[interp] = c.state()
        mask = (c.tags() >= 2) & ((c.tags() == 2) | (np.abs(s) > 1e-9))
        mask[:4, :] = mask[:, :4] = False
        mask[N - 12:, :] = mask[:, N - 12:] = False
        U2 = res[interp]
        np.testing.assert_allclose((U2[1] / U2[0])[mask], u[mask], rtol=0, atol=1e-12)
        np.testing.assert_allclose((U2[2] / U2[0])[mask], v[mask], rtol=0, atol=1e-12)


def test_quadratic_pressure_takes_the_wall_slope_of_an_accelerating_wall(orc):
    """Eq. 5-6 in the quadratic form: the wall slope of the pressure is rho G, G = -n.a_wall, with the density of
    the first probe.  The body oscillates along the wall normal with amplitude h/2; at the end of its stroke
    (t = 1 / (4 f)) the wall lies on the next line of cell centres, is at rest and accelerates by
    -(2 pi f)^2 h / 2 along n.  A pressure field p = p_0 + b s + delta s^2 with b = rho(h) G is then reproduced
    exactly at the IB nodes (all at s = 0, probes at h and 2 h); the same field with the slope left out is not."""
    f = 3.0
    h = math.sqrt(2.0) / N
    spec = dict(_spec(W.INTERP_QUADRATIC), motion=W.MOTION_SIN, amp=(1.0 / (2 * N), 1.0 / (2 * N)), freq=f)
    g, mach = spec["gamma"], spec["mach"]
    R = 1.0 / (g * mach * mach)
    t = 1.0 / (4.0 * f)
    G = (2.0 * math.pi * f) ** 2 * (h / 2.0)  # -n.a_wall
    c = orc.Case(spec)
    c.set_time(t)
    # the two IB nodes where the wall meets the domain's corners have no probe square inside the domain
    assert c.classify() == 2
    xc = (np.arange(N) + 0.5) / N
    X, Y = np.meshgrid(xc, xc)
    s = (X + Y - (C + 1.0 / N)) / math.sqrt(2.0)  # the wall moved by one line of centres
    T = 1.0 + 5.0 * s * s
    Th = 1.0 + 5.0 * h * h
    p0, delta = R, 4.0 * R
    for with_slope in (True, False):
        # p(h) = p0 + b h + delta h^2 with b = G p(h) / (R T(h))
        ph = (p0 + delta * h * h) / (1.0 - G * h / (R * Th)) if with_slope else p0 + delta * h * h
        b = G * ph / (R * Th) if with_slope else 0.0
        p = p0 + b * s + delta * s * s
        u = 0.7 * s - 3.1 * s * s  # the wall is at rest at the end of its stroke
        v = -0.4 * s + 2.3 * s * s
        r = p / (R * T)
        c.set_state(np.stack([r, r * u, r * v, p / (g - 1.0) + 0.5 * r * (u * u + v * v)]))
        c.reconstruct(t)
        U2 = c.state()
        errs = []
        for st in c.stencils(0):
            i, j = st["cell"] % N, st["cell"] // N
            if min(i, j) < 4 or max(i, j) > N - 12:
                continue
            assert abs(s[j, i]) < 1e-12 and abs(st["xi_probe"] - h) < 1e-12
            rr, mx, my, E = U2[:, j, i]
            pp = (g - 1.0) * (E - 0.5 * (mx * mx + my * my) / rr)
            errs.append(abs(pp - p[j, i]) / R)
        assert len(errs) >= 20
        if with_slope:
            assert max(errs) < 1e-11, max(errs)
        else:
            assert min(errs) > 1e-4, min(errs)
