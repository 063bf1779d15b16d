"""ctypes binding of the C ABI in include/ibm.h (argument marshalling only).

Every function of the C ABI is exposed under the same name; ``Case`` wraps a
case handle for convenience.  All computation runs in libibm_gb300.so on the
GPU; there is no CPU path.  Importing this module without the built library
raises at once.
"""
import ctypes
import os

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libibm_gb300.so")

IBM_OK, IBM_EINVAL, IBM_ENOMEM, IBM_ECAPACITY, IBM_ESTENCIL, IBM_ECUDA, IBM_ESTATE = range(7)
(IBM_STATE_FP64, IBM_TAGS, IBM_LIST_COUNTS, IBM_STENCILS, IBM_TIME, IBM_STEPS, IBM_TUNING, IBM_STAGE_LAUNCH,
 IBM_BODY) = range(9)
STATUS_NAMES = {0: "IBM_OK", 1: "IBM_EINVAL", 2: "IBM_ENOMEM", 3: "IBM_ECAPACITY", 4: "IBM_ESTENCIL",
                5: "IBM_ECUDA", 6: "IBM_ESTATE"}


class ibm_geometry(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nverts", ctypes.c_int), ("verts", ctypes.POINTER(ctypes.c_double))]


class ibm_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("lo", ctypes.c_double * 2),
                ("hi", ctypes.c_double * 2), ("bc", ctypes.c_int * 4)]


class ibm_flow(ctypes.Structure):
    _fields_ = [("mach", ctypes.c_double), ("re", ctypes.c_double), ("gamma", ctypes.c_double),
                ("prandtl", ctypes.c_double), ("cfl", ctypes.c_double), ("uinf", ctypes.c_double * 2),
                ("dt_fixed", ctypes.c_double), ("ref_len", ctypes.c_double), ("precision", ctypes.c_int),
                ("time_scheme", ctypes.c_int), ("subiters", ctypes.c_int), ("ib_mode", ctypes.c_int),
                ("dt_phys", ctypes.c_double), ("cfl_tau", ctypes.c_double), ("scheme", ctypes.c_int),
                ("ib_interp", ctypes.c_int)]


class ibm_motion(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("amp", ctypes.c_double * 2), ("freq", ctypes.c_double),
                ("vel", ctypes.c_double * 2), ("mass", ctypes.c_double), ("pivot", ctypes.c_double * 2),
                ("pitch_mean", ctypes.c_double), ("pitch_amp", ctypes.c_double)]


STENCIL_DTYPE = np.dtype([
    ("cell", "<i4"), ("feature", "<i4"), ("region", "<i4"), ("i0", "<i4"), ("j0", "<i4"),
    ("mask", "<i4"), ("nstep", "<i4"), ("kind", "<i4"),
    ("nx", "<f8"), ("ny", "<f8"), ("bx", "<f8"), ("by", "<f8"),
    ("xi_node", "<f8"), ("xi_probe", "<f8"), ("w", "<f8", (4,)), ("curv", "<f8"),
    ("i0b", "<i4"), ("j0b", "<i4"), ("maskb", "<i4"), ("nstepb", "<i4"), ("xi_probe2", "<f8"), ("wb", "<f8", (4,)),
])

class ibm_grid3d(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3)]


CLOSEST3D_DTYPE = np.dtype([("node", "<i4"), ("tri", "<i4"), ("kind", "<i4"), ("reserved", "<i4"),
                            ("cp", "<f8", (3,)), ("n", "<f8", (3,))])
IBM_3D_TAGS, IBM_3D_COUNTS, IBM_3D_NODES, IBM_3D_CLOSEST, IBM_3D_STATE, IBM_3D_STENCILS, IBM_3D_TIME = range(7)


class ibm_flow3d(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3), ("bc", ctypes.c_int * 6), ("mach", ctypes.c_double),
                ("re", ctypes.c_double), ("gamma", ctypes.c_double), ("prandtl", ctypes.c_double),
                ("cfl", ctypes.c_double), ("uinf", ctypes.c_double * 3), ("dt_fixed", ctypes.c_double),
                ("ref_area", ctypes.c_double), ("precision", ctypes.c_int)]


STENCIL3D_DTYPE = np.dtype([
    ("node", "<i4"), ("kind", "<i4"), ("region", "<i4"), ("nstep", "<i4"),
    ("i0", "<i4"), ("j0", "<i4"), ("k0", "<i4"), ("mask", "<i4"),
    ("n", "<f8", (3,)), ("b", "<f8", (3,)), ("xi_node", "<f8"), ("xi_probe", "<f8"), ("w", "<f8", (8,)),
])


class ibm_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("state", ctypes.c_int32), ("status", ctypes.c_int32),
                ("steps_done", ctypes.c_int64), ("t", ctypes.c_double), ("forces", ctypes.c_double * 4),
                ("submit_s", ctypes.c_double), ("start_s", ctypes.c_double), ("finish_s", ctypes.c_double)]


EXPORTS = ["ibm_create_case", "ibm_classify", "ibm_step", "ibm_get_state", "ibm_set_state", "ibm_set_state_async",
           "ibm_forces", "ibm_surface",
           "ibm_sync", "ibm_destroy_case", "ibm_case_device_bytes", "ibm_launch_count", "ibm_last_error",
           "ibm_profile_enable", "ibm_profile_read", "ibm_use_graphs", "ibm_tag_nodes_noalloc",
           "ibm_server_create", "ibm_server_submit", "ibm_server_progress", "ibm_server_poll",
           "ibm_server_destroy", "ibm_server_set_mode", "ibm_server_stats", "ibm_autotune", "ibm_use_tma",
           "ibm_use_persistent", "ibm_persistent_grid", "ibm_stage_launches",
           "ibm_check_float_conversions", "ibm_fma_peak", "ibm_body3d_create", "ibm_body3d_classify",
           "ibm_body3d_get", "ibm_body3d_destroy", "ibm_case3d_create", "ibm_case3d_step", "ibm_case3d_get",
           "ibm_case3d_set_state", "ibm_case3d_forces", "ibm_case3d_launch_count", "ibm_case3d_destroy"]
REQ_PENDING, REQ_RUNNING, REQ_DONE, REQ_FAILED = range(4)
SERVE_BATCHED, SERVE_AUTOTUNE = 1, 2
SERVER_STATS = ["group_graphs", "group_steps", "group_kernels", "autotune_runs", "capture_us"]
PROFILE_GROUPS = ["residual_stage", "ib_reconstruct", "domain_halo", "time_step", "geometry", "step_end"]


class IbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libibm_gb300.so is not built; run __graft_entry__.build() "
                          "(the library has no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    vp, ip, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    L.ibm_create_case.argtypes = [ctypes.POINTER(ibm_geometry), ctypes.POINTER(ibm_grid),
                                  ctypes.POINTER(ibm_flow), ctypes.POINTER(ibm_motion), vp,
                                  ctypes.POINTER(vp)]
    L.ibm_classify.argtypes = [vp]
    L.ibm_step.argtypes = [vp, ip]
    L.ibm_get_state.argtypes = [vp, ip, vp, sz, ip]
    L.ibm_set_state.argtypes = [vp, vp, sz, ip]
    L.ibm_set_state_async.argtypes = [vp, vp, sz, ip]
    L.ibm_forces.argtypes = [vp, vp]
    L.ibm_surface.argtypes = [vp, vp, vp, ip]
    L.ibm_fma_peak.argtypes = [ip, ctypes.c_longlong, vp, vp]
    L.ibm_fma_peak.restype = ip
    L.ibm_body3d_create.argtypes = [vp, ip, vp, ip, vp, vp]
    L.ibm_body3d_classify.argtypes = [vp, vp]
    L.ibm_body3d_get.argtypes = [vp, ip, vp, ctypes.c_size_t]
    L.ibm_body3d_destroy.argtypes = [vp]
    for name in ("ibm_body3d_create", "ibm_body3d_classify", "ibm_body3d_get", "ibm_body3d_destroy"):
        getattr(L, name).restype = ip
    L.ibm_case3d_create.argtypes = [vp, ip, vp, ip, ctypes.POINTER(ibm_flow3d), vp, ctypes.POINTER(vp)]
    L.ibm_case3d_step.argtypes = [vp, ip]
    L.ibm_case3d_get.argtypes = [vp, ip, vp, sz, ip]
    L.ibm_case3d_set_state.argtypes = [vp, vp, sz, ip]
    L.ibm_case3d_forces.argtypes = [vp, vp]
    L.ibm_case3d_destroy.argtypes = [vp]
    for name in ("ibm_case3d_create", "ibm_case3d_step", "ibm_case3d_get", "ibm_case3d_set_state",
                 "ibm_case3d_forces", "ibm_case3d_destroy"):
        getattr(L, name).restype = ip
    L.ibm_case3d_launch_count.argtypes = [vp]
    L.ibm_case3d_launch_count.restype = ctypes.c_int64
    L.ibm_sync.argtypes = [vp]
    L.ibm_destroy_case.argtypes = [vp]
    L.ibm_case_device_bytes.argtypes = [ctypes.POINTER(ibm_geometry), ctypes.POINTER(ibm_grid),
                                        ctypes.POINTER(ibm_flow), ctypes.POINTER(ibm_motion)]
    L.ibm_case_device_bytes.restype = sz
    L.ibm_launch_count.argtypes = [vp]
    L.ibm_launch_count.restype = ctypes.c_int64
    L.ibm_last_error.restype = ctypes.c_char_p
    L.ibm_profile_enable.argtypes = [vp, ip]
    L.ibm_profile_read.argtypes = [vp, vp, vp, ip]
    L.ibm_use_graphs.argtypes = [vp, ip]
    L.ibm_autotune.argtypes = [vp, ip]
    L.ibm_autotune.restype = ip
    L.ibm_use_tma.argtypes = [vp, ip]
    L.ibm_use_tma.restype = ip
    L.ibm_use_persistent.argtypes = [vp, ip]
    L.ibm_use_persistent.restype = ip
    L.ibm_persistent_grid.argtypes = [vp, ip]
    L.ibm_persistent_grid.restype = ip
    L.ibm_stage_launches.argtypes = [vp, ip]
    L.ibm_stage_launches.restype = ip
    L.ibm_check_float_conversions.argtypes = [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]
    L.ibm_check_float_conversions.restype = ip
    L.ibm_tag_nodes_noalloc.argtypes = [ctypes.POINTER(ibm_grid), vp, ip, vp, vp, ctypes.c_int32, vp, vp]
    L.ibm_tag_nodes_noalloc.restype = ip
    L.ibm_server_create.argtypes = [sz, ip, ip, ctypes.POINTER(vp)]
    L.ibm_server_submit.argtypes = [vp, ctypes.POINTER(ibm_geometry), ctypes.POINTER(ibm_grid),
                                    ctypes.POINTER(ibm_flow), ctypes.POINTER(ibm_motion), ip,
                                    ctypes.POINTER(ctypes.c_int64)]
    L.ibm_server_progress.argtypes = [vp, ctypes.POINTER(ip), ctypes.POINTER(ip)]
    L.ibm_server_poll.argtypes = [vp, ctypes.c_int64, ctypes.POINTER(ibm_result)]
    L.ibm_server_destroy.argtypes = [vp]
    L.ibm_server_set_mode.argtypes = [vp, ip]
    L.ibm_server_stats.argtypes = [vp, vp, ip]
    for name in ("ibm_server_create", "ibm_server_submit", "ibm_server_progress", "ibm_server_poll",
                 "ibm_server_destroy", "ibm_server_set_mode", "ibm_server_stats"):
        getattr(L, name).restype = ip
    for name in ("ibm_create_case", "ibm_classify", "ibm_step", "ibm_get_state", "ibm_set_state",
                 "ibm_set_state_async", "ibm_forces", "ibm_surface", "ibm_sync", "ibm_destroy_case", "ibm_profile_enable", "ibm_profile_read",
                 "ibm_use_graphs"):
        getattr(L, name).restype = ip
    return L


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


def _check(status):
    if status != IBM_OK:
        raise IbmError(status, lib().ibm_last_error().decode())
    return status


def marshal(spec):
    """Case spec (workloads.case_spec) -> C structs (kept alive by the returned tuple)."""
    verts = np.ascontiguousarray(spec["verts"], np.float64).reshape(-1, 2)
    geo = ibm_geometry(2, verts.shape[0],
                       verts.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if verts.shape[0] else None)
    gr = ibm_grid()
    gr.nx, gr.ny = spec["nx"], spec["ny"]
    x0, x1, y0, y1 = spec["domain"]
    gr.lo[0], gr.lo[1], gr.hi[0], gr.hi[1] = x0, y0, x1, y1
    for s in range(4):
        gr.bc[s] = spec["bc"][s]
    fl = ibm_flow()
    fl.mach, fl.re, fl.gamma, fl.prandtl, fl.cfl = spec["mach"], spec["re"], spec["gamma"], spec["prandtl"], \
        spec["cfl"]
    fl.uinf[0], fl.uinf[1] = spec["uinf"]
    fl.dt_fixed = spec.get("dt_fixed", 0.0)
    fl.ref_len = spec.get("ref_len", 1.0)
    fl.precision = spec.get("precision", W.PREC_FP64)
    fl.time_scheme = spec.get("time_scheme", W.TIME_RK3)
    fl.subiters = spec.get("subiters", 30)
    fl.dt_phys = spec.get("dt_phys", 0.0)
    fl.cfl_tau = spec.get("cfl_tau", 0.8)
    fl.ib_mode = spec.get("ib_mode", W.IB_REBUILD)
    fl.scheme = spec.get("scheme", W.SCHEME_WENO5)
    fl.ib_interp = spec.get("ib_interp", W.INTERP_LINEAR)
    mo = ibm_motion()
    mo.kind = spec.get("motion", W.MOTION_STATIC)
    mo.amp[0], mo.amp[1] = spec.get("amp", (0.0, 0.0))
    mo.freq = spec.get("freq", 0.0)
    mo.vel[0], mo.vel[1] = spec.get("vel", (0.0, 0.0))
    mo.mass = spec.get("mass", 0.0)
    mo.pivot[0], mo.pivot[1] = spec.get("pivot", (0.0, 0.0))
    mo.pitch_mean = spec.get("pitch_mean", 0.0)
    mo.pitch_amp = spec.get("pitch_amp", 0.0)
    return verts, geo, gr, fl, mo


def fma_peak(fp64, iters):
    """Measured FMA rate of the current device: (flop/s, launch ms) for FP32 (fp64 False) or FP64."""
    f, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib().ibm_fma_peak(int(bool(fp64)), int(iters), ctypes.byref(f), ctypes.byref(ms)))
    return f.value, ms.value


def ibm_tag_nodes_noalloc(spec, d_verts, nverts, d_tags, d_cells, capacity, d_counts, stream=None):
    """Allocation-free tagging (device pointers in, device pointers out); see include/ibm.h."""
    verts, geo, gr, fl, mo = marshal(spec)
    _check(lib().ibm_tag_nodes_noalloc(ctypes.byref(gr), ctypes.c_void_p(d_verts), int(nverts),
                                       ctypes.c_void_p(d_tags), ctypes.c_void_p(d_cells), int(capacity),
                                       ctypes.c_void_p(d_counts), ctypes.c_void_p(stream) if stream else None))


def check_float_conversions():
    """(values compared, mismatches) of the dual-time update's integer-bit FP32 <-> FP64 conversions against the
    hardware conversions on the current device."""
    n, bad = ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(lib().ibm_check_float_conversions(ctypes.byref(n), ctypes.byref(bad)))
    return int(n.value), int(bad.value)


def case_device_bytes(spec):
    verts, geo, gr, fl, mo = marshal(spec)
    return lib().ibm_case_device_bytes(ctypes.byref(geo), ctypes.byref(gr), ctypes.byref(fl), ctypes.byref(mo))


class Case:
    """A solver case on the current CUDA device (owned by the library)."""

    def __init__(self, spec, stream=None):
        self.spec = spec
        self.nx, self.ny = spec["nx"], spec["ny"]
        self._keep = marshal(spec)
        verts, geo, gr, fl, mo = self._keep
        h = ctypes.c_void_p()
        st = ctypes.c_void_p(stream) if stream else None
        _check(lib().ibm_create_case(ctypes.byref(geo), ctypes.byref(gr), ctypes.byref(fl), ctypes.byref(mo), st,
                                     ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().ibm_destroy_case(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def classify(self):
        _check(lib().ibm_classify(self.h))

    def step(self, n=1):
        _check(lib().ibm_step(self.h, int(n)))

    def sync(self):
        _check(lib().ibm_sync(self.h))

    def _get(self, what, arr, on_device=False, ptr=None):
        p = ptr if ptr is not None else arr.ctypes.data_as(ctypes.c_void_p)
        nbytes = arr.nbytes if arr is not None else 0
        _check(lib().ibm_get_state(self.h, what, p, nbytes, 1 if on_device else 0))
        return arr

    def state(self):
        return self._get(IBM_STATE_FP64, np.empty((4, self.ny, self.nx), np.float64))

    def state_to_device(self, tensor):
        """Copy the FP64 state into a CUDA tensor of shape (4, ny, nx), float64."""
        assert tensor.is_cuda and tensor.dtype.itemsize == 8 and tensor.is_contiguous()
        _check(lib().ibm_get_state(self.h, IBM_STATE_FP64, ctypes.c_void_p(tensor.data_ptr()),
                                   tensor.numel() * 8, 1))

    def set_state(self, a):
        a = np.ascontiguousarray(a, np.float64)
        assert a.shape == (4, self.ny, self.nx)
        _check(lib().ibm_set_state(self.h, a.ctypes.data_as(ctypes.c_void_p), a.nbytes, 0))

    def set_state_from_ptr(self, ptr, nbytes, on_device, wait=True):
        """wait=False: ibm_set_state_async (the source must stay unchanged until the next synchronising call)."""
        f = lib().ibm_set_state if wait else lib().ibm_set_state_async
        _check(f(self.h, ctypes.c_void_p(ptr), nbytes, 1 if on_device else 0))

    def tags(self):
        return self._get(IBM_TAGS, np.empty((self.ny, self.nx), np.uint8))

    def counts(self):
        return self._get(IBM_LIST_COUNTS, np.zeros(4, np.int32))

    def stencils(self):
        n = int(self.counts().sum())
        a = np.zeros(n, STENCIL_DTYPE)
        if n:
            self._get(IBM_STENCILS, a)
        return a

    def time(self):
        return self._get(IBM_TIME, np.zeros(2, np.float64))

    def steps(self):
        return int(self._get(IBM_STEPS, np.zeros(1, np.int64))[0])

    def forces(self):
        out = np.zeros(4, np.float64)
        _check(lib().ibm_forces(self.h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def surface(self):
        """Per segment (Eq. 9 integrand at the midpoints): pressure and skin-friction coefficients."""
        n = int(self.spec["verts"].shape[0])
        cp = np.zeros(n, np.float64)
        cf = np.zeros(n, np.float64)
        _check(lib().ibm_surface(self.h, cp.ctypes.data_as(ctypes.c_void_p), cf.ctypes.data_as(ctypes.c_void_p), n))
        return cp, cf

    def forces_into(self, ptr):
        """Forces written to caller memory at ptr (host, 4 doubles)."""
        _check(lib().ibm_forces(self.h, ctypes.c_void_p(ptr)))

    def launches(self):
        return int(lib().ibm_launch_count(self.h))

    def autotune(self, enable):
        _check(lib().ibm_autotune(self.h, int(enable)))

    def stage_launch(self):
        """Launch form of the FP32-bulk stages (0..2; -1 for FP64)."""
        out = np.zeros(1, np.int32)
        _check(lib().ibm_get_state(self.h, IBM_STAGE_LAUNCH, out.ctypes.data_as(ctypes.c_void_p), 4, 0))
        return int(out[0])

    def body(self):
        """Body displacement (x, y), velocity (u, v) and the force per unit depth (Fx, Fy) that set the last
        step's acceleration (motion under the fluid force, Eq. 10; zeros otherwise)."""
        out = np.zeros(6, np.float64)
        _check(lib().ibm_get_state(self.h, IBM_BODY, out.ctypes.data_as(ctypes.c_void_p), out.nbytes, 0))
        return out

    def tuning(self):
        """Register-budget variants of the plain stage kernel: (stage 1, stages 2-3)."""
        out = np.zeros(2, np.int32)
        _check(lib().ibm_get_state(self.h, IBM_TUNING, out.ctypes.data_as(ctypes.c_void_p), 8, 0))
        return int(out[0]), int(out[1])

    def use_tma(self, enable):
        _check(lib().ibm_use_tma(self.h, int(enable)))

    def use_persistent(self, enable):
        _check(lib().ibm_use_persistent(self.h, int(enable)))

    def persistent_grid(self, blocks):
        _check(lib().ibm_persistent_grid(self.h, int(blocks)))

    def stage_launches(self, mode):
        _check(lib().ibm_stage_launches(self.h, int(mode)))

    def use_graphs(self, enable):
        _check(lib().ibm_use_graphs(self.h, 1 if enable else 0))

    def profile(self, enable):
        _check(lib().ibm_profile_enable(self.h, 1 if enable else 0))

    def profile_read(self):
        """{group: (ms, launches)} summed since the last read."""
        n = len(PROFILE_GROUPS)
        ms = np.zeros(n, np.float64)
        cnt = np.zeros(n, np.int64)
        _check(lib().ibm_profile_read(self.h, ms.ctypes.data_as(ctypes.c_void_p), cnt.ctypes.data_as(ctypes.c_void_p),
                                      n))
        return {g: (float(ms[k]), int(cnt[k])) for k, g in enumerate(PROFILE_GROUPS)}


class Server:
    """Request loop over many cases on the current CUDA device (see ibm_server_* in include/ibm.h).

    ``submit`` queues a case spec with a step count; ``progress`` runs one
    non-blocking pass of the native loop (retire, admit, enqueue); ``poll``
    returns the request's record as a dict.
    """

    def __init__(self, device_bytes_budget=0, max_active=16, steps_per_chunk=10,
                 mode=SERVE_BATCHED | SERVE_AUTOTUNE):
        h = ctypes.c_void_p()
        _check(lib().ibm_server_create(int(device_bytes_budget), int(max_active), int(steps_per_chunk),
                                       ctypes.byref(h)))
        self.h = h
        _check(lib().ibm_server_set_mode(self.h, int(mode)))

    def stats(self):
        out = np.zeros(len(SERVER_STATS), np.int64)
        _check(lib().ibm_server_stats(self.h, out.ctypes.data_as(ctypes.c_void_p), len(SERVER_STATS)))
        return dict(zip(SERVER_STATS, (int(v) for v in out)))

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            lib().ibm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, spec, nsteps):
        verts, geo, gr, fl, mo = marshal(spec)
        rid = ctypes.c_int64()
        _check(lib().ibm_server_submit(self.h, ctypes.byref(geo), ctypes.byref(gr), ctypes.byref(fl),
                                       ctypes.byref(mo), int(nsteps), ctypes.byref(rid)))
        return rid.value

    def progress(self):
        na, npend = ctypes.c_int(), ctypes.c_int()
        _check(lib().ibm_server_progress(self.h, ctypes.byref(na), ctypes.byref(npend)))
        return na.value, npend.value

    def poll(self, rid):
        r = ibm_result()
        _check(lib().ibm_server_poll(self.h, int(rid), ctypes.byref(r)))
        return dict(id=r.id, state=r.state, status=r.status, steps_done=r.steps_done, t=r.t,
                    forces=np.array(r.forces[:], np.float64), submit_s=r.submit_s, start_s=r.start_s,
                    finish_s=r.finish_s)

    def drain(self, sleep_s=0.0):
        """Run the loop until no request is running or waiting."""
        import time
        while True:
            na, npend = self.progress()
            if na == 0 and npend == 0:
                return
            if sleep_s:
                time.sleep(sleep_s)


class Body3D:
    """A closed triangulated surface on the device (ibm_body3d_*): 3-D classification, tagging, ordered lists
    and closest features with pseudo-normals on a uniform lattice (Sec. 3.2, 4.1-4.2)."""

    def __init__(self, verts, tris, stream=None):
        self.verts = np.ascontiguousarray(verts, np.float64).reshape(-1, 3)
        self.tris = np.ascontiguousarray(tris, np.int32).reshape(-1, 3)
        h = ctypes.c_void_p()
        _check(lib().ibm_body3d_create(self.verts.ctypes.data_as(ctypes.c_void_p), self.verts.shape[0],
                                       self.tris.ctypes.data_as(ctypes.c_void_p), self.tris.shape[0],
                                       ctypes.c_void_p(stream) if stream else None, ctypes.byref(h)))
        self.h = h
        self.shape = None

    def classify(self, n, lo, hi):
        """n = (nx, ny, nz) lattice nodes over [lo, hi] (asynchronous)."""
        g = ibm_grid3d(int(n[0]), int(n[1]), int(n[2]), (ctypes.c_double * 3)(*lo), (ctypes.c_double * 3)(*hi))
        _check(lib().ibm_body3d_classify(self.h, ctypes.byref(g)))
        self.shape = (int(n[2]), int(n[1]), int(n[0]))

    def _get(self, what, arr):
        _check(lib().ibm_body3d_get(self.h, what, arr.ctypes.data_as(ctypes.c_void_p), arr.nbytes))
        return arr

    def tags(self):
        return self._get(IBM_3D_TAGS, np.empty(self.shape, np.uint8))

    def counts(self):
        return self._get(IBM_3D_COUNTS, np.zeros(4, np.int32))

    def nodes(self):
        return self._get(IBM_3D_NODES, np.zeros(int(self.counts().sum()), np.int32))

    def closest(self):
        return self._get(IBM_3D_CLOSEST, np.zeros(int(self.counts().sum()), CLOSEST3D_DTYPE))

    def close(self):
        if getattr(self, "h", None):
            lib().ibm_body3d_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()


class Case3D:
    """A 3-D case (ibm_case3d_*): a static closed triangulated body in a uniform block, FP64 SSP-RK3 steps.
    ``spec`` is a dict from ``workloads.case3d_spec``."""

    def __init__(self, spec, stream=None):
        self.spec = spec
        self.n = tuple(spec["n"])
        self.verts = np.ascontiguousarray(spec["verts"], np.float64).reshape(-1, 3)
        self.tris = np.ascontiguousarray(spec["tris"], np.int32).reshape(-1, 3)
        f = ibm_flow3d()
        f.nx, f.ny, f.nz = self.n
        for a in range(3):
            f.lo[a], f.hi[a], f.uinf[a] = spec["lo"][a], spec["hi"][a], spec["uinf"][a]
        for k in range(6):
            f.bc[k] = spec["bc"][k]
        f.mach, f.re, f.gamma, f.prandtl, f.cfl = spec["mach"], spec["re"], spec["gamma"], spec["prandtl"], spec["cfl"]
        f.dt_fixed, f.ref_area = spec["dt_fixed"], spec["ref_area"]
        f.precision = spec.get("precision", W.PREC_FP64)
        self._flow = f
        h = ctypes.c_void_p()
        _check(lib().ibm_case3d_create(self.verts.ctypes.data_as(ctypes.c_void_p), self.verts.shape[0],
                                       self.tris.ctypes.data_as(ctypes.c_void_p), self.tris.shape[0],
                                       ctypes.byref(f), ctypes.c_void_p(stream) if stream else None,
                                       ctypes.byref(h)))
        self.h = h
        self.shape = (self.n[2], self.n[1], self.n[0])

    def step(self, n=1):
        _check(lib().ibm_case3d_step(self.h, int(n)))

    def _get(self, what, arr):
        _check(lib().ibm_case3d_get(self.h, what, arr.ctypes.data_as(ctypes.c_void_p), arr.nbytes, 0))
        return arr

    def state(self):
        return self._get(IBM_3D_STATE, np.empty((5,) + self.shape, np.float64))

    def set_state(self, a):
        a = np.ascontiguousarray(a, np.float64)
        assert a.shape == (5,) + self.shape
        _check(lib().ibm_case3d_set_state(self.h, a.ctypes.data_as(ctypes.c_void_p), a.nbytes, 0))

    def tags(self):
        return self._get(IBM_3D_TAGS, np.empty(self.shape, np.uint8))

    def counts(self):
        return self._get(IBM_3D_COUNTS, np.zeros(4, np.int32))

    def stencils(self):
        return self._get(IBM_3D_STENCILS, np.zeros(int(self.counts().sum()), STENCIL3D_DTYPE))

    def time(self):
        return self._get(IBM_3D_TIME, np.zeros(2, np.float64))

    def forces(self):
        out = np.zeros(6, np.float64)
        _check(lib().ibm_case3d_forces(self.h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def launches(self):
        return int(lib().ibm_case3d_launch_count(self.h))

    def close(self):
        if getattr(self, "h", None):
            lib().ibm_case3d_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()
