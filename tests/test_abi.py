"""The C-ABI library loads and exports every entry point include/lsd.h declares (no GPU).

Only host-side behaviour is exercised here: symbol export, status strings and argument
validation that happens before any CUDA call.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lsd.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+char\s*\*|int)\s+(lsd_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lsdlib():
    from paper_2406_18655_gb300 import build
    build.build()
    from paper_2406_18655_gb300 import lsd
    return lsd


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("lsd_create", "lsd_decode_batch", "lsd_postprocess_batch", "lsd_destroy",
                     "lsd_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lsdlib):
    L = lsdlib.lib()
    for name in _declared():
        assert hasattr(L, name), name
    assert set(_declared()) <= set(lsdlib.EXPORTS)


def test_status_strings(lsdlib):
    assert lsdlib.status_string(0) == "ok"
    assert "budget" in lsdlib.status_string(lsdlib.LSD_ERR_ADMISSION)
    assert "image" in lsdlib.status_string(lsdlib.SHOT_UNSOLVABLE)


def test_create_rejects_bad_arguments_before_touching_the_gpu(lsdlib):
    L = lsdlib.lib()
    h = C.c_void_p()
    rows = np.array([0, 0, 1], np.int32)
    cols = np.array([0, 1, 1], np.int32)
    p = np.full(2, 0.1, np.float32)
    P = lambda a: a.ctypes.data_as(C.c_void_p)
    # m < 1
    assert L.lsd_create(C.byref(h), 0, 2, 3, P(rows), P(cols), P(p), 10, 0, None) == -1
    # index out of range
    bad = np.array([0, 0, 5], np.int32)
    assert L.lsd_create(C.byref(h), 2, 2, 3, P(bad), P(cols), P(p), 10, 0, None) == -1
    # duplicate entry
    dup_r = np.array([0, 0], np.int32)
    dup_c = np.array([1, 1], np.int32)
    assert L.lsd_create(C.byref(h), 2, 2, 2, P(dup_r), P(dup_c), P(p), 10, 0, None) == -1
    # probability outside (0, 1)
    badp = np.array([0.1, 1.5], np.float32)
    assert L.lsd_create(C.byref(h), 2, 2, 3, P(rows), P(cols), P(badp), 10, 0, None) == -1
    # LSD order beyond the limit
    assert L.lsd_create(C.byref(h), 2, 2, 3, P(rows), P(cols), P(p), 10, 99, None) == -1
    # nonzero reserved option
    opt = lsdlib.Options()
    opt.reserved = 1
    assert L.lsd_create(C.byref(h), 2, 2, 3, P(rows), P(cols), P(p), 10, 0, C.byref(opt)) == -1
    # OSD-CS: sweep order beyond 8, a sweep order without the sweep, an unknown method, and
    # growth beyond 65535 steps
    for method, w, order in ((1, 9, 4), (0, 2, 4), (2, 0, 4), (1, 4, 65536)):
        opt = lsdlib.Options()
        opt.osd_method, opt.osd_cs_order = method, w
        assert L.lsd_create(C.byref(h), 2, 2, 3, P(rows), P(cols), P(p), 10, order,
                            C.byref(opt)) == -1
    assert not h.value
    # window decoder: commit beyond the window, no rounds, an index out of range
    pq = np.full(2, 0.1, np.float32)
    for d, w, c, r in ((3, 3, 4, rows), (0, 3, 1, rows), (3, 0, 1, rows), (3, 3, 0, rows),
                       (3, 3, 1, bad)):
        assert L.lsd_window_create(C.byref(h), 2, 2, 3, P(r), P(cols), P(pq), P(pq), d, w, c, 10,
                                   0, None) == -1
    assert L.lsd_window_destroy(None) == 0
    # giant-shot decoder: no edges, a bad index, a bad probability
    for r, c, pp, nnz in ((rows, cols, p, 0), (bad, cols, p, 3), (rows, cols, badp, 3)):
        assert L.lsd_giant_create(C.byref(h), 2, 2, nnz, P(r), P(c), P(pp), 10, 0, 0, None) == -1
    assert L.lsd_giant_create(C.byref(h), 2, 2, 3, P(rows), P(cols), P(p), 10, 13, 0, None) == -1
    assert L.lsd_giant_destroy(None) == 0
    assert L.lsd_giant_decode(None, None, None, None, None) == -1
    assert L.lsd_window_decode(None, 1, None, None, None, None) == -1
    # NULL handles are rejected or ignored
    assert L.lsd_destroy(None) == 0
    assert L.lsd_decode_batch(None, 1, None, None, None, None, None) == -1


def test_bp_variant_names(lsdlib):
    """Variant ids of the autotuner's report name the kernel and shape that ran (host only)."""
    names = [lsdlib.bp_variant_name(v) for v in range(64)]
    assert names[2] == "bp_kernel<32,0>"
    assert names[7] == "bp_reg_kernel<32,3,6,5,3>"
    assert any(n.startswith("bp_regcta_kernel<128,3,8,6,3,true,6>") for n in names)
    assert lsdlib.bp_variant_name(-1) == "" and names[-1] == ""
