"""FP64 CPU oracle (ctypes wrapper over ``oracle.c`` and, for the 3-D flow, ``oracle3d.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU-baseline
leg of the benchmark are the only callers.  The CUDA library never imports,
links or executes anything in this directory, and this directory shares no code
with it; the two meet only through the seeded inputs built by
``paper_1912_11908_gb300.workloads`` (geometry vertices and case parameters,
which hold none of the method's arithmetic).
"""
import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboracle.so")
SOURCES = [os.path.join(HERE, "oracle.c"), os.path.join(HERE, "oracle3d.c")]

FLUID, SOLID, IB, G1, G2, G3 = range(6)
BC_FREESTREAM, BC_OUTFLOW, BC_PERIODIC = range(3)
MOTION_STATIC, MOTION_SIN, MOTION_CONST, MOTION_COUPLED, MOTION_PITCH = range(5)


def build(force=False):
    """Compile the oracle with gcc (IEEE binary64, no FMA contraction)."""
    newest = max(os.path.getmtime(s) for s in SOURCES + [os.path.join(HERE, "oracle.h")])
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= newest:
        return LIB_PATH
    tmp = LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-fPIC", "-shared", "-o", tmp] + SOURCES + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double), ("y0", ctypes.c_double), ("y1", ctypes.c_double),
        ("bc", ctypes.c_int * 4),
        ("mach", ctypes.c_double), ("re", ctypes.c_double), ("gamma", ctypes.c_double),
        ("prandtl", ctypes.c_double), ("cfl", ctypes.c_double),
        ("uinf", ctypes.c_double * 2), ("dt_fixed", ctypes.c_double), ("ref_len", ctypes.c_double),
        ("nv", ctypes.c_int), ("verts", ctypes.POINTER(ctypes.c_double)),
        ("motion", ctypes.c_int), ("amp", ctypes.c_double * 2), ("freq", ctypes.c_double),
        ("vel", ctypes.c_double * 2), ("mass", ctypes.c_double), ("ib_mode", ctypes.c_int),
        ("pivot", ctypes.c_double * 2), ("pitch_mean", ctypes.c_double), ("pitch_amp", ctypes.c_double),
        ("scheme", ctypes.c_int),
        ("time_scheme", ctypes.c_int), ("subiters", ctypes.c_int), ("dt_phys", ctypes.c_double),
        ("cfl_tau", ctypes.c_double), ("ib_interp", ctypes.c_int),
    ]


class _Params3(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3), ("bc", ctypes.c_int * 6),
        ("mach", ctypes.c_double), ("re", ctypes.c_double), ("gamma", ctypes.c_double),
        ("prandtl", ctypes.c_double), ("cfl", ctypes.c_double),
        ("uinf", ctypes.c_double * 3), ("dt_fixed", ctypes.c_double), ("ref_area", ctypes.c_double),
        ("nv", ctypes.c_int), ("ntri", ctypes.c_int),
        ("verts", ctypes.POINTER(ctypes.c_double)), ("tris", ctypes.POINTER(ctypes.c_int)),
    ]


STENCIL3_DTYPE = np.dtype([
    ("node", "<i4"), ("kind", "<i4"), ("region", "<i4"), ("nstep", "<i4"),
    ("i0", "<i4"), ("j0", "<i4"), ("k0", "<i4"), ("mask", "<i4"),
    ("n", "<f8", (3,)), ("b", "<f8", (3,)), ("xi_node", "<f8"), ("xi_probe", "<f8"), ("w", "<f8", (8,)),
])

STENCIL_DTYPE = np.dtype([
    ("cell", "<i4"), ("feature", "<i4"), ("region", "<i4"), ("i0", "<i4"), ("j0", "<i4"),
    ("mask", "<i4"), ("nstep", "<i4"), ("kind", "<i4"),
    ("nx", "<f8"), ("ny", "<f8"), ("bx", "<f8"), ("by", "<f8"),
    ("xi_node", "<f8"), ("xi_probe", "<f8"), ("w", "<f8", (4,)), ("curv", "<f8"),
    ("i0b", "<i4"), ("j0b", "<i4"), ("maskb", "<i4"), ("nstepb", "<i4"), ("xi_probe2", "<f8"), ("wb", "<f8", (4,)),
])

_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB_PATH)
        vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.orc_create.restype = vp
        L.orc_create.argtypes = [ctypes.POINTER(_Params)]
        L.orc_destroy.argtypes = [vp]
        L.orc_classify.argtypes = [vp]
        L.orc_classify.restype = ip
        L.orc_step.argtypes = [vp, ip]
        L.orc_step.restype = ip
        L.orc_get_state.argtypes = [vp, vp]
        L.orc_set_state.argtypes = [vp, vp]
        L.orc_set_time.argtypes = [vp, dp]
        L.orc_get_tags.argtypes = [vp, vp]
        L.orc_list_len.argtypes = [vp, ip]
        L.orc_list_len.restype = ip
        L.orc_get_list.argtypes = [vp, ip, vp]
        L.orc_forces.argtypes = [vp, vp]
        L.orc_surface.argtypes = [vp, vp, vp]
        L.orc_body.argtypes = [vp, vp]
        L.orc_time.argtypes = [vp]
        L.orc_time.restype = dp
        L.orc_last_dt.argtypes = [vp]
        L.orc_last_dt.restype = dp
        L.orc_reconstruct.argtypes = [vp, dp]
        L.orc_vertex_normals.argtypes = [vp, vp]
        L.orc_closest.argtypes = [vp, dp, dp, vp, vp, vp, vp, vp]
        L.orc_classify_points.argtypes = [ip, vp, ip, vp, vp]
        L.orc_classify_points_3d.argtypes = [ip, vp, ip, vp, ip, vp, vp]
        L.orc_closest_3d.argtypes = [ip, vp, ip, vp, ip, vp, vp, vp, vp]
        L.orc_tags_3d.argtypes = [ip, ip, ip, vp, vp]
        L.orc_weno5.argtypes = [vp]
        L.orc_tvd2.argtypes = [vp]
        L.orc_tvd2.restype = dp
        L.orc_weno5.restype = dp
        L.orc_ldfss_xflux.argtypes = [vp, vp, dp, dp, dp, vp]
        L.orc_euler_xflux.argtypes = [vp, dp, dp, vp]
        L.orc_precond_matrix.argtypes = [vp, dp, dp, dp, vp]
        L.orc_dwdq.argtypes = [vp, dp, dp, vp]
        L.orc_solve4.argtypes = [vp, vp, vp]
        L.orc_solve4.restype = ip
        L.orc3_create.restype = vp
        L.orc3_create.argtypes = [ctypes.POINTER(_Params3)]
        L.orc3_destroy.argtypes = [vp]
        L.orc3_classify.argtypes = [vp]
        L.orc3_classify.restype = ip
        L.orc3_step.argtypes = [vp, ip]
        L.orc3_step.restype = ip
        L.orc3_reconstruct.argtypes = [vp]
        L.orc3_get_state.argtypes = [vp, vp]
        L.orc3_set_state.argtypes = [vp, vp]
        L.orc3_get_tags.argtypes = [vp, vp]
        L.orc3_list_len.argtypes = [vp, ip]
        L.orc3_list_len.restype = ip
        L.orc3_get_list.argtypes = [vp, ip, vp]
        L.orc3_forces.argtypes = [vp, vp]
        L.orc3_time.argtypes = [vp]
        L.orc3_time.restype = dp
        L.orc3_last_dt.argtypes = [vp]
        L.orc3_last_dt.restype = dp
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class Case:
    """One oracle case; ``spec`` is a dict from ``workloads.case_spec``."""

    def __init__(self, spec):
        s = spec
        self.spec = spec
        self.nx, self.ny = s["nx"], s["ny"]
        verts = np.ascontiguousarray(s.get("verts", np.zeros((0, 2))), dtype=np.float64).reshape(-1, 2)
        self._verts = verts
        P = _Params()
        P.nx, P.ny = s["nx"], s["ny"]
        P.x0, P.x1, P.y0, P.y1 = s["domain"]
        for k in range(4):
            P.bc[k] = s["bc"][k]
        P.mach, P.re, P.gamma, P.prandtl, P.cfl = s["mach"], s["re"], s["gamma"], s["prandtl"], s["cfl"]
        P.uinf[0], P.uinf[1] = s["uinf"]
        P.dt_fixed = s.get("dt_fixed", 0.0)
        P.ref_len = s.get("ref_len", 1.0)
        P.nv = verts.shape[0]
        P.verts = verts.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if P.nv else None
        P.motion = s.get("motion", MOTION_STATIC)
        amp = s.get("amp", (0.0, 0.0))
        vel = s.get("vel", (0.0, 0.0))
        P.amp[0], P.amp[1] = amp
        P.freq = s.get("freq", 0.0)
        P.vel[0], P.vel[1] = vel
        P.mass = s.get("mass", 0.0)
        P.ib_mode = s.get("ib_mode", 0)
        P.pivot[0], P.pivot[1] = s.get("pivot", (0.0, 0.0))
        P.pitch_mean = s.get("pitch_mean", 0.0)
        P.pitch_amp = s.get("pitch_amp", 0.0)
        P.scheme = s.get("scheme", 0)
        P.time_scheme = s.get("time_scheme", 0)
        P.subiters = s.get("subiters", 30)
        P.dt_phys = s.get("dt_phys", 0.0)
        P.cfl_tau = s.get("cfl_tau", 0.8)
        P.ib_interp = s.get("ib_interp", 0)
        self._P = P
        self.h = lib().orc_create(ctypes.byref(P))

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    def classify(self):
        return lib().orc_classify(self.h)

    def step(self, n):
        return lib().orc_step(self.h, n)

    def state(self):
        a = np.empty((4, self.ny, self.nx), np.float64)
        lib().orc_get_state(self.h, _ptr(a))
        return a

    def set_state(self, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        assert a.shape == (4, self.ny, self.nx)
        lib().orc_set_state(self.h, _ptr(a))

    def set_time(self, t):
        lib().orc_set_time(self.h, float(t))

    def tags(self):
        a = np.empty((self.ny, self.nx), np.uint8)
        lib().orc_get_tags(self.h, _ptr(a))
        return a

    def stencils(self, kind):
        n = lib().orc_list_len(self.h, kind)
        a = np.zeros(n, STENCIL_DTYPE)
        if n:
            lib().orc_get_list(self.h, kind, _ptr(a))
        return a

    def forces(self):
        out = np.zeros(4, np.float64)
        lib().orc_forces(self.h, _ptr(out))
        return out

    def surface(self):
        """Per segment (Eq. 9 integrand at the midpoints): pressure coefficient (p_s - p_inf) / (rho U^2 / 2)
        and skin-friction coefficient tau / (rho U^2 / 2); NaN where no probe square was found."""
        n = self._verts.shape[0]
        cp = np.zeros(n, np.float64)
        cf = np.zeros(n, np.float64)
        lib().orc_surface(self.h, _ptr(cp), _ptr(cf))
        return cp, cf

    def time(self):
        return lib().orc_time(self.h)

    def body(self):
        """Body displacement (x, y), velocity (u, v) and the force per unit depth (Fx, Fy) that set the last
        step's acceleration (coupled motion, Eq. 10)."""
        out = np.zeros(6, np.float64)
        lib().orc_body(self.h, _ptr(out))
        return out

    def last_dt(self):
        return lib().orc_last_dt(self.h)

    def reconstruct(self, t):
        lib().orc_reconstruct(self.h, t)

    def vertex_normals(self):
        a = np.zeros((self._verts.shape[0], 2), np.float64)
        lib().orc_vertex_normals(self.h, _ptr(a))
        return a

    def closest(self, x, y):
        f = ctypes.c_int32()
        r = ctypes.c_int32()
        cx, cy, d2 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        lib().orc_closest(self.h, x, y, ctypes.byref(f), ctypes.byref(r), ctypes.byref(cx), ctypes.byref(cy),
                          ctypes.byref(d2))
        return f.value, r.value, cx.value, cy.value, d2.value


class Case3D:
    """One 3-D oracle case (static closed triangulated body, SSP-RK3); ``spec`` is a dict from
    ``workloads.case3d_spec``."""

    def __init__(self, spec):
        s = spec
        self.spec = spec
        self.nx, self.ny, self.nz = s["n"]
        self._verts = np.ascontiguousarray(s["verts"], np.float64).reshape(-1, 3)
        self._tris = np.ascontiguousarray(s["tris"], np.int32).reshape(-1, 3)
        P = _Params3()
        P.nx, P.ny, P.nz = s["n"]
        for a in range(3):
            P.lo[a], P.hi[a] = s["lo"][a], s["hi"][a]
            P.uinf[a] = s["uinf"][a]
        for k in range(6):
            P.bc[k] = s["bc"][k]
        P.mach, P.re, P.gamma, P.prandtl, P.cfl = s["mach"], s["re"], s["gamma"], s["prandtl"], s["cfl"]
        P.dt_fixed = s["dt_fixed"]
        P.ref_area = s["ref_area"]
        P.nv, P.ntri = self._verts.shape[0], self._tris.shape[0]
        if P.ntri:
            P.verts = self._verts.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            P.tris = self._tris.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        self._P = P
        self.h = lib().orc3_create(ctypes.byref(P))

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc3_destroy(self.h)
            self.h = None

    def classify(self):
        return lib().orc3_classify(self.h)

    def step(self, n):
        return lib().orc3_step(self.h, n)

    def reconstruct(self):
        lib().orc3_reconstruct(self.h)

    def state(self):
        a = np.empty((5, self.nz, self.ny, self.nx), np.float64)
        lib().orc3_get_state(self.h, _ptr(a))
        return a

    def set_state(self, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        assert a.shape == (5, self.nz, self.ny, self.nx)
        lib().orc3_set_state(self.h, _ptr(a))

    def tags(self):
        a = np.empty((self.nz, self.ny, self.nx), np.uint8)
        lib().orc3_get_tags(self.h, _ptr(a))
        return a

    def stencils(self, kind=None):
        """The stencils of one list (0 IB, 1..3 G1..G3), or of all four in that order."""
        if kind is None:
            return np.concatenate([self.stencils(k) for k in range(4)])
        n = lib().orc3_list_len(self.h, kind)
        a = np.zeros(n, STENCIL3_DTYPE)
        if n:
            lib().orc3_get_list(self.h, kind, _ptr(a))
        return a

    def forces(self):
        out = np.zeros(6, np.float64)
        lib().orc3_forces(self.h, _ptr(out))
        return out

    def time(self):
        return lib().orc3_time(self.h)

    def last_dt(self):
        return lib().orc3_last_dt(self.h)


def classify_points_3d(verts, tris, pts):
    """Ray-casting classification against a closed triangulated surface (1 = solid)."""
    verts = np.ascontiguousarray(verts, np.float64).reshape(-1, 3)
    tris = np.ascontiguousarray(tris, np.int32).reshape(-1, 3)
    pts = np.ascontiguousarray(pts, np.float64).reshape(-1, 3)
    out = np.zeros(pts.shape[0], np.uint8)
    lib().orc_classify_points_3d(verts.shape[0], _ptr(verts), tris.shape[0], _ptr(tris), pts.shape[0], _ptr(pts),
                                 _ptr(out))
    return out


def tags_3d(solid):
    """Node tags of a [nz][ny][nx] lattice from its solid flags (IB = fluid with a solid 6-neighbour, G1..G3)."""
    solid = np.ascontiguousarray(solid, np.uint8)
    nz, ny, nx = solid.shape
    out = np.zeros_like(solid)
    lib().orc_tags_3d(nx, ny, nz, _ptr(solid), _ptr(out))
    return out


def closest_3d(verts, tris, pts):
    """Closest surface point, its pseudo-normal and the feature kind (0 face, 1 edge, 2 vertex) per point."""
    verts = np.ascontiguousarray(verts, np.float64).reshape(-1, 3)
    tris = np.ascontiguousarray(tris, np.int32).reshape(-1, 3)
    pts = np.ascontiguousarray(pts, np.float64).reshape(-1, 3)
    cp = np.zeros_like(pts)
    nrm = np.zeros_like(pts)
    kind = np.zeros(pts.shape[0], np.int32)
    lib().orc_closest_3d(verts.shape[0], _ptr(verts), tris.shape[0], _ptr(tris), pts.shape[0], _ptr(pts), _ptr(cp),
                         _ptr(nrm), _ptr(kind))
    return cp, nrm, kind


def classify_points(verts, pts):
    verts = np.ascontiguousarray(verts, np.float64).reshape(-1, 2)
    pts = np.ascontiguousarray(pts, np.float64).reshape(-1, 2)
    out = np.zeros(pts.shape[0], np.uint8)
    lib().orc_classify_points(verts.shape[0], _ptr(verts), pts.shape[0], _ptr(pts), _ptr(out))
    return out


def weno5(f):
    f = np.ascontiguousarray(f, np.float64)
    return lib().orc_weno5(_ptr(f))


def tvd2(f):
    f = np.ascontiguousarray(f, np.float64)
    return lib().orc_tvd2(_ptr(f))


def ldfss_xflux(qL, qR, gamma, R, mr2=1.0):
    qL = np.ascontiguousarray(qL, np.float64)
    qR = np.ascontiguousarray(qR, np.float64)
    F = np.zeros(4)
    lib().orc_ldfss_xflux(_ptr(qL), _ptr(qR), gamma, R, mr2, _ptr(F))
    return F


def euler_xflux(q, gamma, R):
    q = np.ascontiguousarray(q, np.float64)
    F = np.zeros(4)
    lib().orc_euler_xflux(_ptr(q), gamma, R, _ptr(F))
    return F


def precond_matrix(Q, gamma, R, Ur):
    Q = np.ascontiguousarray(Q, np.float64)
    out = np.zeros(16)
    lib().orc_precond_matrix(_ptr(Q), gamma, R, Ur, _ptr(out))
    return out.reshape(4, 4)


def dwdq(Q, gamma, R):
    Q = np.ascontiguousarray(Q, np.float64)
    out = np.zeros(16)
    lib().orc_dwdq(_ptr(Q), gamma, R, _ptr(out))
    return out.reshape(4, 4)


def solve4(A, b):
    A = np.ascontiguousarray(A, np.float64).ravel()
    b = np.ascontiguousarray(b, np.float64)
    x = np.zeros(4)
    rc = lib().orc_solve4(_ptr(A), _ptr(b), _ptr(x))
    return x if rc == 0 else None
