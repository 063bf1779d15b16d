"""The allocation-free tagging entry point against the case-based one.

ibm_tag_nodes_noalloc serves callers that cannot allocate device memory (it
keeps its intermediate data in a fixed device array inside the library).  Its
tags, list counts and row-major IB / ghost cell lists must equal those of
ibm_classify bit for bit -- the same bar as every tag and list test -- on two
calls in a row with different bodies and grids (the shared array keeps the
previous call's contents).  This file sorts last so a stop-at-first-failure
run has already run every other test.
"""
import numpy as np
import pytest

from paper_1912_11908_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1912_11908_gb300 import _build, ibm
    _build.build()
    ibm.lib()
    return torch, ibm


def _reference(ibm, spec):
    c = ibm.Case(spec)
    c.classify()
    tags = c.tags()
    counts = c.counts()
    cells = c.stencils()["cell"]
    c.close()
    return tags, counts, cells


def test_noalloc_tagging_matches_classify_twice(env):
    torch, ibm = env
    specs = [W.naca0012_a5_m0001(1024, 512, time_scheme=W.TIME_RK3), W.cylinder_m02_re40(150, 70)]
    stream = torch.cuda.current_stream()
    for spec in specs:  # two calls in a row through the shared scratch array
        tags_ref, counts_ref, cells_ref = _reference(ibm, spec)
        nx, ny = spec["nx"], spec["ny"]
        verts = torch.tensor(np.ascontiguousarray(spec["verts"]).ravel(), dtype=torch.float64, device="cuda")
        tags = torch.full((ny, nx), 255, dtype=torch.uint8, device="cuda")
        cap = int(counts_ref.sum()) + 64
        cells = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
        counts = torch.zeros(4, dtype=torch.int32, device="cuda")
        ibm.ibm_tag_nodes_noalloc(spec, verts.data_ptr(), spec["verts"].shape[0], tags.data_ptr(),
                                  cells.data_ptr(), cap, counts.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(tags.cpu().numpy(), tags_ref)
        np.testing.assert_array_equal(counts.cpu().numpy(), counts_ref)
        n = int(counts_ref.sum())
        np.testing.assert_array_equal(cells.cpu().numpy()[:n], cells_ref)
        assert (cells.cpu().numpy()[n:] == -1).all()


def test_noalloc_list_overflow_keeps_totals(env):
    """Capacity below the number of listed nodes: d_counts still holds the full totals, the first `capacity`
    entries are the reference list's, and nothing past capacity is written (a guard region stays untouched)."""
    torch, ibm = env
    spec = W.cylinder_m02_re40(150, 70)
    tags_ref, counts_ref, cells_ref = _reference(ibm, spec)
    n = int(counts_ref.sum())
    cap = n // 2
    guard = 256
    verts = torch.tensor(np.ascontiguousarray(spec["verts"]).ravel(), dtype=torch.float64, device="cuda")
    tags = torch.full((spec["ny"], spec["nx"]), 255, dtype=torch.uint8, device="cuda")
    cells = torch.full((cap + guard,), -7, dtype=torch.int32, device="cuda")
    counts = torch.zeros(4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    ibm.ibm_tag_nodes_noalloc(spec, verts.data_ptr(), spec["verts"].shape[0], tags.data_ptr(), cells.data_ptr(),
                              cap, counts.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(counts.cpu().numpy(), counts_ref)
    np.testing.assert_array_equal(tags.cpu().numpy(), tags_ref)
    out = cells.cpu().numpy()
    np.testing.assert_array_equal(out[:cap], cells_ref[:cap])
    assert (out[cap:] == -7).all()


def test_noalloc_rejects_oversize(env):
    torch, ibm = env
    spec = W.cylinder_m02_re40(4096, 2048)  # 8.4 M cells > 4,194,304
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(ibm.IbmError) as e:
        ibm.ibm_tag_nodes_noalloc(spec, dummy.data_ptr(), 256, dummy.data_ptr(), dummy.data_ptr(), 1,
                                  dummy.data_ptr())
    assert e.value.status == ibm.IBM_EINVAL
