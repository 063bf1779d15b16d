"""CPU-side checks of the C ABI: the library loads, exports every entry point the
header declares, and rejects bad arguments before touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1912_11908_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ibm():
    from paper_1912_11908_gb300 import _build, ibm as mod
    _build.build()
    return mod


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(ibm_\w+)\s*\(", txt, re.M))
    return names


def test_library_exports_every_declared_symbol(ibm):
    L = ibm.lib()
    declared = _declared()
    assert {"ibm_create_case", "ibm_classify", "ibm_step", "ibm_get_state", "ibm_forces",
            "ibm_destroy_case"} <= declared
    for name in sorted(declared):
        assert hasattr(L, name), name
    assert set(ibm.EXPORTS) <= declared


def test_invalid_arguments_rejected_without_gpu(ibm):
    L = ibm.lib()
    spec = W.cylinder_m02_re40(64, 32)
    for bad in (dict(spec, nx=4), dict(spec, mach=0.0), dict(spec, bc=(2, 0, 0, 0)), dict(spec, gamma=1.0),
                dict(spec, precision=7), dict(spec, verts=spec["verts"][:2])):
        verts, geo, gr, fl, mo = ibm.marshal(bad)
        h = ctypes.c_void_p()
        st = L.ibm_create_case(ctypes.byref(geo), ctypes.byref(gr), ctypes.byref(fl), ctypes.byref(mo), None,
                               ctypes.byref(h))
        assert st == ibm.IBM_EINVAL, bad
        assert not h.value
        assert L.ibm_last_error()
    assert L.ibm_destroy_case(None) == ibm.IBM_OK


def test_device_bytes_estimate(ibm):
    fp64 = ibm.case_device_bytes(W.wedge_m2_re1e4())
    fp32 = ibm.case_device_bytes(W.wedge_m2_re1e4(precision=W.PREC_FP32_BULK))
    cells = 768 * 384
    assert 96 * cells < fp64 < 140 * cells
    assert fp32 < fp64


def test_coupled_motion_arguments_rejected_without_gpu(ibm):
    """A body moving under the fluid force needs a positive mass, the explicit scheme and a body; an unknown
    motion kind and a pitching motion without a body are rejected too."""
    L = ibm.lib()
    spec = W.shock_driven_cylinder(64, 64)
    for bad in (dict(spec, mass=0.0), dict(spec, mass=-1.0), dict(spec, time_scheme=W.TIME_DUAL, dt_phys=0.01),
                dict(spec, verts=np.zeros((0, 2))), dict(spec, motion=99),
                dict(spec, motion=W.MOTION_PITCH, verts=np.zeros((0, 2)))):
        verts, geo, gr, fl, mo = ibm.marshal(bad)
        h = ctypes.c_void_p()
        st = L.ibm_create_case(ctypes.byref(geo), ctypes.byref(gr), ctypes.byref(fl), ctypes.byref(mo), None,
                               ctypes.byref(h))
        assert st == ibm.IBM_EINVAL, bad
        assert not h.value


def _header_enums():
    txt = open(os.path.join(ROOT, "include", "ibm.h")).read()
    out = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", txt, re.S):
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        for name, val in re.findall(r"(IBM_\w+)\s*=\s*(\d+)", body):
            out[name] = int(val)
    return out


def test_header_constants_match_the_binding(ibm):
    """Every enum value the binding and the input generators use equals the header's."""
    h = _header_enums()
    for name in ("IBM_OK", "IBM_EINVAL", "IBM_ECAPACITY", "IBM_ESTENCIL", "IBM_STATE_FP64", "IBM_TAGS",
                 "IBM_LIST_COUNTS", "IBM_STENCILS", "IBM_TIME", "IBM_STEPS", "IBM_TUNING", "IBM_STAGE_LAUNCH",
                 "IBM_BODY"):
        assert getattr(ibm, name) == h[name], name
    pairs = {"MOTION_STATIC": "IBM_MOTION_STATIC", "MOTION_SIN": "IBM_MOTION_SIN", "MOTION_CONST": "IBM_MOTION_CONST",
             "MOTION_COUPLED": "IBM_MOTION_COUPLED", "PREC_FP64": "IBM_PREC_FP64",
             "PREC_FP32_BULK": "IBM_PREC_FP32_BULK", "TIME_RK3": "IBM_TIME_RK3", "TIME_DUAL": "IBM_TIME_DUAL",
             "BC_FREESTREAM": "IBM_BC_FREESTREAM", "BC_OUTFLOW": "IBM_BC_OUTFLOW", "BC_PERIODIC": "IBM_BC_PERIODIC",
             "IB_REBUILD": "IBM_IB_REBUILD", "IB_ADVANCE": "IBM_IB_ADVANCE", "MOTION_PITCH": "IBM_MOTION_PITCH",
             "SCHEME_WENO5": "IBM_SCHEME_WENO5", "SCHEME_TVD2": "IBM_SCHEME_TVD2",
             "INTERP_LINEAR": "IBM_INTERP_LINEAR", "INTERP_QUADRATIC": "IBM_INTERP_QUADRATIC"}
    for py, c in pairs.items():
        assert getattr(W, py) == h[c], py
    for name in ("IBM_3D_TAGS", "IBM_3D_COUNTS", "IBM_3D_NODES", "IBM_3D_CLOSEST", "IBM_3D_STATE",
                 "IBM_3D_STENCILS", "IBM_3D_TIME"):
        assert getattr(ibm, name) == h[name], name


def test_struct_layouts_match_the_header(ibm, tmp_path):
    """sizeof and field offsets of the ABI structs, as a C compiler lays them out from the header, equal the
    binding's ctypes layouts (a field added on one side only fails here)."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    structs = {"ibm_geometry": ibm.ibm_geometry, "ibm_grid": ibm.ibm_grid, "ibm_flow": ibm.ibm_flow,
               "ibm_motion": ibm.ibm_motion, "ibm_result": ibm.ibm_result, "ibm_grid3d": ibm.ibm_grid3d,
               "ibm_flow3d": ibm.ibm_flow3d}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ibm.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append('  printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for f in cls._fields_:
            lines.append('  printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, f[0], name, f[0]))
    for f in ibm.STENCIL_DTYPE.names:  # the stencil record is read into a numpy structured array
        lines.append('  printf("ibm_stencil.%s %%zu\\n", offsetof(ibm_stencil, %s));' % (f, f))
    lines.append('  printf("ibm_stencil %zu\\n", sizeof(ibm_stencil));')
    for f in ibm.STENCIL3D_DTYPE.names:
        lines.append('  printf("ibm_stencil3d.%s %%zu\\n", offsetof(ibm_stencil3d, %s));' % (f, f))
    lines.append('  printf("ibm_stencil3d %zu\\n", sizeof(ibm_stencil3d));')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)]).decode().splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f in cls._fields_:
            assert int(got["%s.%s" % (name, f[0])]) == getattr(cls, f[0]).offset, (name, f[0])
    assert int(got["ibm_stencil"]) == ibm.STENCIL_DTYPE.itemsize
    for f in ibm.STENCIL_DTYPE.names:
        assert int(got["ibm_stencil.%s" % f]) == ibm.STENCIL_DTYPE.fields[f][1], f
    assert int(got["ibm_stencil3d"]) == ibm.STENCIL3D_DTYPE.itemsize
    for f in ibm.STENCIL3D_DTYPE.names:
        assert int(got["ibm_stencil3d.%s" % f]) == ibm.STENCIL3D_DTYPE.fields[f][1], f


def test_unknown_reconstruction_rejected(ibm):
    """ibm_flow.scheme other than WENO5 / TVD-2, and ib_interp other than linear / quadratic, are refused by
    the library (no silent default)."""
    L = ibm.lib()
    for bad in (dict(scheme=7), dict(ib_interp=5), dict(ib_interp=-1)):
        verts, geo, gr, fl, mo = ibm.marshal(dict(W.cylinder_m02_re40(64, 32), **bad))
        h = ctypes.c_void_p()
        st = L.ibm_create_case(ctypes.byref(geo), ctypes.byref(gr), ctypes.byref(fl), ctypes.byref(mo), None,
                               ctypes.byref(h))
        assert st == ibm.IBM_EINVAL and not h.value, bad


def test_case3d_arguments_rejected_before_device_work(ibm):
    """ibm_case3d_create refuses malformed cases with IBM_EINVAL and returns no case, before any device call (so
    this runs without a GPU): fewer than 4 cells along an axis, an unknown boundary condition, periodic on one
    side of an axis only, an unknown precision, a non-positive Mach number or reference area, a mesh pointer
    missing for a non-empty mesh."""
    L = ibm.lib()
    good = W.case3d_spec(None, None, (8, 8, 8), (0, 0, 0), (1, 1, 1), 0.3, 100.0, W.FAR3D)
    bads = [dict(n=(3, 8, 8)), dict(bc=(0, 1, 0, 0, 0, 9)), dict(bc=(2, 1, 0, 0, 0, 0)), dict(precision=3),
            dict(mach=0.0), dict(ref_area=0.0)]
    for bad in bads:
        s = dict(good, **bad)
        f = ibm.ibm_flow3d()
        f.nx, f.ny, f.nz = s["n"]
        for a in range(3):
            f.lo[a], f.hi[a], f.uinf[a] = s["lo"][a], s["hi"][a], s["uinf"][a]
        for k in range(6):
            f.bc[k] = s["bc"][k]
        f.mach, f.re, f.gamma, f.prandtl, f.cfl = s["mach"], s["re"], s["gamma"], s["prandtl"], s["cfl"]
        f.dt_fixed, f.ref_area, f.precision = s["dt_fixed"], s["ref_area"], s["precision"]
        h = ctypes.c_void_p()
        st = L.ibm_case3d_create(None, 0, None, 0, ctypes.byref(f), None, ctypes.byref(h))
        assert st == ibm.IBM_EINVAL and not h.value, bad
    f = ibm.ibm_flow3d()
    f.nx = f.ny = f.nz = 8
    for a in range(3):
        f.lo[a], f.hi[a] = 0.0, 1.0
    f.mach, f.gamma, f.prandtl, f.cfl, f.ref_area = 0.3, 1.4, 0.72, 0.5, 1.0
    h = ctypes.c_void_p()
    assert L.ibm_case3d_create(None, 8, None, 12, ctypes.byref(f), None, ctypes.byref(h)) == ibm.IBM_EINVAL
    assert not h.value
