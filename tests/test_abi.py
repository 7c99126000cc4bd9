"""The C-ABI library builds, loads and exports every entry point include/leg.h
declares; argument validation answers without touching a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2311_18482_gb300 import build
    path = build.build()
    return C.CDLL(path)


def _declared():
    text = open(os.path.join(ROOT, "include", "leg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(le_[a-z0-9_]+)\s*\(", text)))


def test_header_symbols_exported(lib):
    names = _declared()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2311_18482_gb300 import binding
    assert set(_declared()) <= set(binding.exported_symbols())


def test_invalid_arguments_rejected_on_host(lib):
    from paper_2311_18482_gb300 import binding as b
    lib.le_last_error.restype = C.c_char_p
    ws = C.c_size_t()
    assert lib.le_bin_sort_workspace(C.c_int32(-1), C.c_int64(10), C.byref(ws)) == b.LE_ERR_INVALID_ARG
    assert lib.le_bin_sort_workspace(C.c_int32(1000), C.c_int64(1 << 33), C.byref(ws)) == b.LE_ERR_INVALID_ARG
    assert lib.le_bin_sort_workspace(C.c_int32(1000), C.c_int64(20000), C.byref(ws)) == b.LE_OK
    assert ws.value >= 2 * 8 * 1000          # two depth-sort buffers of n keys at least
    # null gaussians / camera
    assert lib.le_preprocess(None, None, None, None) == b.LE_ERR_INVALID_ARG
    assert b"null" in lib.le_last_error()
    cam = b.LeCamera()
    cam.width, cam.height, cam.fx, cam.fy = 0, 10, 1.0, 1.0
    g = b.LeGaussians()
    g.n, g.sh_degree = 0, 0
    p = b.LeProjected()
    assert lib.le_preprocess(C.byref(g), C.byref(cam), C.byref(p), None) == b.LE_ERR_INVALID_ARG
    cam.width = 10
    g.sh_degree = 4
    assert lib.le_preprocess(C.byref(g), C.byref(cam), C.byref(p), None) == b.LE_ERR_INVALID_ARG
    # fused backward + Adam: null camera / config rejected before any GPU work
    assert lib.le_render_bwd_adam(None, None, None, None, None, None, None, None, None, None, None, None, None,
                                  None, None) == b.LE_ERR_INVALID_ARG
    # the projection Adam with an extra range: negative size, unaligned extra pointer
    cam.width, cam.height = 16, 16
    g.n, g.sh_degree = 0, 0
    cfg = b.LeAdamConfig(1, 1e-3, 0.9, 0.999, 1e-8)
    f = lib.le_project_bwd_adam_extra
    args = (C.byref(cam), C.byref(g), C.byref(p), None, None, None, C.byref(cfg))
    assert f(*args, C.c_void_p(16), C.c_void_p(16), C.c_void_p(32), C.c_void_p(48), C.c_int64(-1),
             None) == b.LE_ERR_INVALID_ARG
    assert f(*args, C.c_void_p(18), C.c_void_p(16), C.c_void_p(32), C.c_void_p(48), C.c_int64(8),
             None) == b.LE_ERR_INVALID_ARG
    assert b"aligned" in lib.le_last_error()
    assert f(*args, None, None, None, None, C.c_int64(0), None) == b.LE_OK      # nothing to do
    # misaligned Adam buffers
    assert lib.le_adam(C.c_int64(8), C.c_void_p(3), C.c_void_p(16), C.c_void_p(32), C.c_void_p(48), 1,
                       C.c_float(1e-3), C.c_float(0.9), C.c_float(0.999), C.c_float(1e-8), C.c_float(0),
                       C.c_float(1), None) == b.LE_ERR_INVALID_ARG
    assert lib.le_adam(C.c_int64(8), C.c_void_p(16), C.c_void_p(16), C.c_void_p(32), C.c_void_p(48), 0,
                       C.c_float(1e-3), C.c_float(0.9), C.c_float(0.999), C.c_float(1e-8), C.c_float(0),
                       C.c_float(1), None) == b.LE_ERR_INVALID_ARG
