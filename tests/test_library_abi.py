"""CPU-side checks of the C ABI: the library loads, exports every entry point the
header declares, and rejects bad arguments before touching a GPU."""
import ctypes
import os
import re

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
