"""Seeded synthetic inputs: body polylines and case parameters.

This module is the only code shared by the CUDA path's callers and the CPU
oracle's callers.  It builds inputs only (closed-form body shapes, grid and
flow parameters, request mixes) and contains none of the method's arithmetic.

Bodies are closed counter-clockwise polylines (interior on the left of the
travel direction), the 2-D form of the paper's closed oriented surface
(Sec. 3.1).  Non-dimensional free stream: density 1, temperature 1, reference
speed 1 along +x, reference length 1 (cylinder diameter, chord).
"""
import math

import numpy as np

BC_FREESTREAM, BC_OUTFLOW, BC_PERIODIC = 0, 1, 2
MOTION_STATIC, MOTION_SIN, MOTION_CONST, MOTION_COUPLED, MOTION_PITCH = 0, 1, 2, 3, 4
PREC_FP64, PREC_FP32_BULK = 0, 1
IB_REBUILD, IB_ADVANCE = 0, 1
SCHEME_WENO5, SCHEME_TVD2 = 0, 1
INTERP_LINEAR, INTERP_QUADRATIC = 0, 1  # IB / ghost reconstruction along the normal (ibm_flow.ib_interp)
TIME_RK3, TIME_DUAL = 0, 1


def cylinder(n=256, diameter=1.0, center=(0.0, 0.0)):
    """Regular n-gon inscribed in the circle of the given diameter (Sec. 8.1.1, 8.2.2)."""
    k = np.arange(n, dtype=np.float64)
    a = 2.0 * math.pi * k / n
    r = 0.5 * diameter
    return np.stack([center[0] + r * np.cos(a), center[1] + r * np.sin(a)], axis=1)


def naca00xx(thickness=0.12, n=400, alpha_deg=0.0, chord=1.0):
    """Symmetric NACA 4-digit section with the closed (sharp) trailing edge.

    Half thickness y_t = 5 t (0.2969 sqrt(x) - 0.1260 x - 0.3516 x^2 + 0.2843 x^3
    - 0.1036 x^4); cosine spacing; one trailing-edge vertex, leading edge at the
    origin; rotated nose-up by alpha about the leading edge so that the free
    stream stays along +x (Sec. 7.1, 8.1.2).  n must be even.
    """
    assert n % 2 == 0
    m = n // 2
    k = np.arange(m + 1, dtype=np.float64)
    x = 0.5 * (1.0 - np.cos(math.pi * k / m))
    yt = 5.0 * thickness * (0.2969 * np.sqrt(x) - 0.1260 * x - 0.3516 * x ** 2 + 0.2843 * x ** 3 - 0.1036 * x ** 4)
    yt[0] = 0.0
    yt[-1] = 0.0
    # trailing edge -> upper surface -> leading edge -> lower surface (CCW)
    upper = np.stack([x[::-1], yt[::-1]], axis=1)[:-1]      # k = m .. 1
    lower = np.stack([x[:-1], -yt[:-1]], axis=1)             # k = 0 .. m-1
    pts = np.concatenate([upper, lower], axis=0) * chord
    a = math.radians(alpha_deg)
    ca, sa = math.cos(a), math.sin(a)
    rot = np.stack([pts[:, 0] * ca + pts[:, 1] * sa, -pts[:, 0] * sa + pts[:, 1] * ca], axis=1)
    return rot


def wedge(half_angle_deg=15.0, chord=1.0):
    """Wedge with its apex at the origin pointing upstream (Sec. 8.1.6)."""
    t = math.tan(math.radians(half_angle_deg)) * chord
    return np.array([[0.0, 0.0], [chord, -t], [chord, t]], dtype=np.float64)


def case_spec(verts, nx, ny, domain, mach, re, bc, *, cfl=0.5, uinf=(1.0, 0.0), gamma=1.4, prandtl=0.72,
              motion=MOTION_STATIC, amp=(0.0, 0.0), freq=0.0, vel=(0.0, 0.0), mass=0.0, dt_fixed=0.0, ref_len=1.0,
              precision=PREC_FP64, time_scheme=TIME_RK3, subiters=30, dt_phys=0.0, cfl_tau=0.8, ib_mode=IB_REBUILD,
              scheme=SCHEME_WENO5, ib_interp=INTERP_LINEAR, name=""):
    verts = np.zeros((0, 2)) if verts is None else np.ascontiguousarray(verts, np.float64)
    return dict(name=name, verts=verts, nx=int(nx), ny=int(ny), domain=tuple(float(v) for v in domain),
                mach=float(mach), re=float(re), bc=tuple(int(b) for b in bc), cfl=float(cfl),
                uinf=tuple(float(u) for u in uinf), gamma=float(gamma), prandtl=float(prandtl),
                motion=int(motion), amp=tuple(float(a) for a in amp), freq=float(freq),
                vel=tuple(float(v) for v in vel), mass=float(mass), dt_fixed=float(dt_fixed), ref_len=float(ref_len),
                precision=int(precision), time_scheme=int(time_scheme), subiters=int(subiters),
                dt_phys=float(dt_phys), cfl_tau=float(cfl_tau), ib_mode=int(ib_mode), scheme=int(scheme),
                ib_interp=int(ib_interp))


FAR = (BC_FREESTREAM, BC_OUTFLOW, BC_FREESTREAM, BC_FREESTREAM)
SUPERSONIC = (BC_FREESTREAM, BC_OUTFLOW, BC_OUTFLOW, BC_OUTFLOW)
PERIODIC = (BC_PERIODIC,) * 4


def cylinder_m02_re40(nx=160, ny=80, **kw):
    """Stationary cylinder, 256 segments, M=0.2, Re=40, 160x80 cells over [-8,24]x[-8,8]; 200 RK3 steps."""
    return case_spec(cylinder(256), nx, ny, (-8.0, 24.0, -8.0, 8.0), 0.2, 40.0, FAR,
                     name="cylinder_M0.2_Re40_%dx%d" % (nx, ny), **kw)


def wedge_m2_re1e4(nx=768, ny=384, **kw):
    """15 deg half-angle wedge, chord 1, M=2, Re=1e4, 768x384 cells over [-1,3]x[-1,1]; 2000 RK3 steps.  IB nodes
    are advanced by the flux update and the wall is imposed by the ghost layers (IB_ADVANCE): rebuilt from their
    probes every stage, they discard the mass the supersonic stream carries into them."""
    kw.setdefault("ib_mode", IB_ADVANCE)
    return case_spec(wedge(15.0), nx, ny, (-1.0, 3.0, -1.0, 1.0), 2.0, 1.0e4, SUPERSONIC,
                     name="wedge15_M2_Re1e4_%dx%d" % (nx, ny), **kw)


def oscillating_cylinder_m02_re185(nx=1024, ny=512, **kw):
    """Cylinder oscillating transversely, y(t)=0.2 sin(2 pi 0.16 t), M=0.2, Re=185, 1024x512 over [-10,30]x[-10,10]."""
    return case_spec(cylinder(256), nx, ny, (-10.0, 30.0, -10.0, 10.0), 0.2, 185.0, FAR, motion=MOTION_SIN,
                     amp=(0.0, 0.2), freq=0.16, name="osc_cylinder_M0.2_Re185_%dx%d" % (nx, ny), **kw)


def moving_cylinder_supersonic(mach_d=1.2, nx=3200, ny=640, length=80.0, height=16.0, start=1.5, **kw):
    """Cylinder moving at constant supersonic speed through gas at rest (Sec. 8.2.3): speed 1 along -x, Mach
    and Reynolds numbers (300) on that speed, domain length x height diameters, centre `start` diameters from
    the right side at mid-height; the wake leaves through the left side, the bow shock through the top and
    bottom (zero-gradient), the gas ahead is at rest.  The paper's case runs along +x on a stretched grid with
    D/80 near the body; this one uses a uniform grid (D/40 by default)."""
    verts = cylinder(256, 1.0, center=(length - start, 0.5 * height))
    bc = (BC_OUTFLOW, BC_FREESTREAM, BC_OUTFLOW, BC_OUTFLOW)
    return case_spec(verts, nx, ny, (0.0, length, 0.0, height), mach_d, 300.0, bc, uinf=(0.0, 0.0),
                     motion=MOTION_CONST, vel=(-1.0, 0.0), name="moving_cylinder_M%g_Re300_%dx%d" % (mach_d, nx, ny),
                     **kw)


def stationary_cylinder_supersonic(mach_d=1.2, nx=1600, ny=640, length=40.0, height=16.0, upstream=8.0, **kw):
    """Galilean counterpart of moving_cylinder_supersonic: the cylinder at rest, the stream at speed 1 along +x
    at the same Mach and Reynolds numbers; `upstream` diameters of domain ahead of the centre."""
    verts = cylinder(256, 1.0, center=(upstream, 0.5 * height))
    return case_spec(verts, nx, ny, (0.0, length, 0.0, height), mach_d, 300.0, SUPERSONIC,
                     name="stationary_cylinder_M%g_Re300_%dx%d" % (mach_d, nx, ny), **kw)


def shock_driven_cylinder(nx=656, ny=656, mach_s=1.5, density_ratio=10.0, shock_x=0.5, **kw):
    """Planar shock driving a cylinder free to translate (Sec. 8.2.6), in diameters (D = 0.1 m) and in units of
    the pre-shock gas (density 1, sound speed 1: reference Mach 1, gas at rest).  Domain 4 x 4 diameters
    (0.4 m), centre (1.5, 2) D, D/164 on the paper's 656 x 656 grid; shock Mach 1.5 starting at x = 0.5 D and
    moving along +x; inviscid.  The cylinder's mass per unit depth is density_ratio times that of the gas it
    displaces.  Sides: zero-gradient behind the shock (left) and across it (bottom, top), gas at rest ahead."""
    verts = cylinder(256, 1.0, center=(1.5, 2.0))
    spec = case_spec(verts, nx, ny, (0.0, 4.0, 0.0, 4.0), 1.0, 0.0, (BC_OUTFLOW, BC_FREESTREAM, BC_OUTFLOW, BC_OUTFLOW),
                     uinf=(0.0, 0.0), motion=MOTION_COUPLED, mass=density_ratio * math.pi * 0.25,
                     name="shock_driven_cylinder_Ms%g_%dx%d" % (mach_s, nx, ny), **kw)
    spec["shock"] = (float(shock_x), float(mach_s))
    return spec


def shock_initial_state(spec):
    """Conserved state [4][ny][nx] of a planar shock at x = x_s moving along +x at Mach M_s into gas at rest
    (density 1, pressure p_inf = 1 / (gamma M^2) of the spec): the Rankine-Hugoniot state behind it,
    rho1 = (g+1) Ms^2 / ((g-1) Ms^2 + 2), p1 = p_inf (1 + 2g (Ms^2 - 1) / (g+1)), u1 = Ms c (1 - 1/rho1)."""
    xs, ms = spec["shock"]
    g = spec["gamma"]
    p0 = 1.0 / (g * spec["mach"] ** 2)
    c0 = math.sqrt(g * p0)
    r1 = (g + 1.0) * ms * ms / ((g - 1.0) * ms * ms + 2.0)
    p1 = p0 * (1.0 + 2.0 * g * (ms * ms - 1.0) / (g + 1.0))
    u1 = ms * c0 * (1.0 - 1.0 / r1)
    nx, ny = spec["nx"], spec["ny"]
    x0, x1, _, _ = spec["domain"]
    xc = x0 + (np.arange(nx) + 0.5) * (x1 - x0) / nx
    behind = np.broadcast_to(xc < xs, (ny, nx))
    r = np.where(behind, r1, 1.0)
    u = np.where(behind, u1, 0.0)
    p = np.where(behind, p1, p0)
    return np.stack([r, r * u, np.zeros_like(r), p / (g - 1.0) + 0.5 * r * u * u])


def pitching_naca0012(nx=425, ny=317, mean_deg=30.0, amp_deg=15.0, freq=0.1, mach=0.006, re=3000.0, **kw):
    """NACA0012 pitching about mid-chord (Sec. 7.2): alpha(t) = mean - amp cos(2 pi f t), reduced frequency
    f* = f C / U = 0.1, Re 3000, M 0.006, domain 40C x 30C on the paper's 425 x 317 nodes (here uniform cells).
    The vertices are the airfoil at alpha = 0; the pose rotates them about the pivot (0.5, 0).  Dual time
    (explicit steps would be acoustically limited at this Mach number)."""
    kw.setdefault("time_scheme", TIME_DUAL)
    kw.setdefault("dt_phys", 0.5 * 40.0 / nx)
    spec = case_spec(naca00xx(0.12, 400, 0.0), nx, ny, (-10.0, 30.0, -15.0, 15.0), mach, re, FAR,
                     motion=MOTION_PITCH, freq=freq, name="pitching_naca0012_%dx%d" % (nx, ny), **kw)
    spec.update(pivot=(0.5, 0.0), pitch_mean=math.radians(mean_deg), pitch_amp=math.radians(amp_deg))
    return spec


def naca0012_a5_m0001(nx=2048, ny=1024, **kw):
    """NACA0012 at 5 deg, 400 vertices, M=0.001, Re=1000, 2048x1024 over [-4,8]x[-3,3]; dual time, 30 sub-iterations."""
    dx = 12.0 / nx
    kw.setdefault("time_scheme", TIME_DUAL)
    kw.setdefault("dt_phys", 0.5 * dx)
    return case_spec(naca00xx(0.12, 400, 5.0), nx, ny, (-4.0, 8.0, -3.0, 3.0), 0.001, 1000.0, FAR,
                     name="naca0012_a5_M0.001_Re1000_%dx%d" % (nx, ny), **kw)


def uv_sphere(n_lat=21, n_lon=30, radius=1.0, center=(0.0, 0.0, 0.0)):
    """Closed triangulated sphere (Appendix A: 1200 triangles for 21 x 30): two poles and n_lat - 1 rings of
    n_lon vertices; triangles counter-clockwise seen from outside."""
    verts = [(0.0, 0.0, radius)]
    for i in range(1, n_lat):
        th = math.pi * i / n_lat
        for j in range(n_lon):
            ph = 2.0 * math.pi * j / n_lon
            verts.append((radius * math.sin(th) * math.cos(ph), radius * math.sin(th) * math.sin(ph),
                          radius * math.cos(th)))
    verts.append((0.0, 0.0, -radius))
    south = len(verts) - 1
    ring = lambda i, j: 1 + (i - 1) * n_lon + (j % n_lon)  # noqa: E731
    tris = []
    for j in range(n_lon):
        tris.append((0, ring(1, j), ring(1, j + 1)))
    for i in range(1, n_lat - 1):
        for j in range(n_lon):
            a, b, c, d = ring(i, j), ring(i, j + 1), ring(i + 1, j), ring(i + 1, j + 1)
            tris.append((a, c, d))
            tris.append((a, d, b))
    for j in range(n_lon):
        tris.append((south, ring(n_lat - 1, j + 1), ring(n_lat - 1, j)))
    return np.array(verts) + np.array(center), np.array(tris, dtype=np.int32)


def box_mesh(lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    """Closed triangulated box: 8 corners, two triangles per face, counter-clockwise seen from outside (sharp
    edges and corners for the pseudo-normal checks of Sec. 4.2)."""
    x0, y0, z0 = lo
    x1, y1, z1 = hi
    verts = np.array([(x0, y0, z0), (x1, y0, z0), (x1, y1, z0), (x0, y1, z0),
                      (x0, y0, z1), (x1, y0, z1), (x1, y1, z1), (x0, y1, z1)], dtype=np.float64)
    quads = [(0, 3, 2, 1), (4, 5, 6, 7), (0, 1, 5, 4), (2, 3, 7, 6), (1, 2, 6, 5), (0, 4, 7, 3)]
    tris = []
    for a, b, c, d in quads:
        tris += [(a, b, c), (a, c, d)]
    return verts, np.array(tris, dtype=np.int32)


def case3d_spec(verts, tris, n, lo, hi, mach, re, bc, *, cfl=0.5, uinf=(1.0, 0.0, 0.0), gamma=1.4, prandtl=0.72,
                dt_fixed=0.0, ref_area=1.0, precision=PREC_FP64, name=""):
    """A 3-D case: nx * ny * nz cells over [lo, hi], a static closed triangulated body (verts None: no body),
    domain sides in the order x-low, x-high, y-low, y-high, z-low, z-high."""
    if verts is None:
        verts, tris = np.zeros((0, 3)), np.zeros((0, 3), np.int32)
    return dict(name=name, verts=np.ascontiguousarray(verts, np.float64).reshape(-1, 3),
                tris=np.ascontiguousarray(tris, np.int32).reshape(-1, 3), n=tuple(int(v) for v in n),
                lo=tuple(float(v) for v in lo), hi=tuple(float(v) for v in hi), mach=float(mach), re=float(re),
                bc=tuple(int(b) for b in bc), cfl=float(cfl), uinf=tuple(float(u) for u in uinf), gamma=float(gamma),
                prandtl=float(prandtl), dt_fixed=float(dt_fixed), ref_area=float(ref_area),
                precision=int(precision))


FAR3D = (BC_FREESTREAM, BC_OUTFLOW) + (BC_FREESTREAM,) * 4


def sphere_m03_re100(nx=192, ny=96, nz=96, **kw):
    """Flow past the Appendix A sphere (UV sphere of 1200 triangles), diameter 1 at the origin, M 0.3, Re 100
    (steady axisymmetric wake), over [-3, 9] x [-3, 3] x [-3, 3]; forces normalised by the frontal area."""
    verts, tris = uv_sphere(radius=0.5)
    return case3d_spec(verts, tris, (nx, ny, nz), (-3.0, -3.0, -3.0), (9.0, 3.0, 3.0), 0.3, 100.0, FAR3D,
                       ref_area=math.pi * 0.25, name="sphere_M0.3_Re100_%dx%dx%d" % (nx, ny, nz), **kw)


def random_polygon(rng, n, center=(0.0, 0.0), rmin=0.3, rmax=1.0):
    """Star-shaped random polygon (CCW) for brute-force classification checks."""
    a = np.sort(rng.uniform(0.0, 2.0 * math.pi, n))
    r = rng.uniform(rmin, rmax, n)
    return np.stack([center[0] + r * np.cos(a), center[1] + r * np.sin(a)], axis=1)


def serving_mix(n=512, seed=20191224, mean_interarrival_s=0.05, nsteps=500, dual_mach=0.01, dual_steps=10,
                subiters=30):
    """Request mix for the request loop: bodies, motions, Mach, Re and grids drawn from a seed.

    Each entry: arrival time (Poisson process), case spec (FP32-bulk) and the
    number of steps the request asks for: `nsteps` explicit SSP-RK3 steps, or,
    at M <= dual_mach, `dual_steps` dual-time physical steps of dt = 0.5 h with
    `subiters` sub-iterations (explicit steps would be acoustically limited).
    """
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(mean_interarrival_s, n))
    reqs = []
    nxs = [64, 128, 256, 512, 1024]
    nys = [64, 128, 256, 512]
    pairs = [(a, b) for a in nxs for b in nys if b <= a]
    for k in range(n):
        body = int(rng.integers(0, 3))
        osc = bool(rng.integers(0, 2))
        mach = float(math.exp(rng.uniform(math.log(0.001), math.log(2.0))))
        re = float(math.exp(rng.uniform(math.log(40.0), math.log(1.0e4))))
        gx, gy = pairs[int(rng.integers(0, len(pairs)))]
        if body == 0:
            verts = cylinder(256)
        elif body == 1:
            verts = naca00xx(float(rng.uniform(0.09, 0.15)), 400, 0.0)
        else:
            verts = wedge(float(rng.uniform(10.0, 20.0)))
        # square cells; at least 12 body lengths along x and 3 across, body 4 lengths from the inflow
        h = max(12.0 / gx, 3.0 / gy)
        dom = (-4.0, -4.0 + gx * h, -0.5 * gy * h, 0.5 * gy * h)
        dual = mach <= dual_mach
        kw = dict(time_scheme=TIME_DUAL, dt_phys=0.5 * h, subiters=subiters) if dual else {}
        reqs.append(dict(arrival_s=float(t[k]), nsteps=int(dual_steps if dual else nsteps), spec=case_spec(
            verts, gx, gy, dom, mach, re, FAR if mach < 1.0 else SUPERSONIC,
            motion=MOTION_SIN if osc else MOTION_STATIC, amp=(0.0, 0.2) if osc else (0.0, 0.0),
            freq=0.16 if osc else 0.0, precision=PREC_FP32_BULK, name="req%03d" % k, **kw)))
    return reqs
