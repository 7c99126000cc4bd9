"""le_bin_sort_static: the binning entry point for callers that cannot
allocate device memory -- code that runs inside a host application or plugin
whose device memory belongs to someone else, or a per-frame path that cannot
take cudaMalloc's implicit synchronisation.  Its scratch is a static array
inside the library.

Two calls in a row, through the C ABI, on different scenes: each must give
exactly the sorted ids, 64-bit keys, tile ranges and K of le_bin_sort with a
caller workspace (binning is integer work, so the bar is bit-exactness).  The
second call also shows that what the first left in the shared array does not
leak into it.  A repeated call is checked to take no device memory: neither
PyTorch's allocator nor the driver's free-memory count moves across it.  This
file is named to be collected last.
"""
import numpy as np
import pytest
import torch

from paper_2311_18482_gb300 import synth

pytestmark = pytest.mark.gpu


def _project(leg, name, **kw):
    c = synth.config(name, **kw)
    cam = c["camera"]
    g = leg.Gaussians.from_scene(c["scene"])
    return cam, leg.le_preprocess(g, cam)


def test_static_scratch_matches_workspace_path(leg):
    for name, kw in (("c2", dict(n=20000, W=320, H=240)), ("c1", {})):
        cam, proj = _project(leg, name, **kw)
        ids_ws, ranges_ws, K_ws, keys_ws = leg.le_bin_sort(cam, proj, want_keys=True)
        ids_ws, ranges_ws, keys_ws = ids_ws.clone(), ranges_ws.clone(), keys_ws.clone()
        assert 0 < K_ws <= 524288
        cap = K_ws + 100
        ids = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
        keys = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
        ranges = torch.full_like(ranges_ws, -1)
        K = leg.le_bin_sort_static(cam, proj, ids, ranges, keys)
        torch.cuda.synchronize()
        assert K == K_ws
        assert torch.equal(ids[:K], ids_ws)
        assert torch.equal(keys[:K], keys_ws)
        assert torch.equal(ranges, ranges_ws)


def test_static_scratch_allocates_nothing(leg):
    cam, proj = _project(leg, "c2", n=20000, W=320, H=240)
    _, _, K_ws, _ = leg.le_bin_sort(cam, proj)
    ids = torch.empty(K_ws, dtype=torch.int32, device="cuda")
    ranges = torch.empty((cam.tiles_x * cam.tiles_y, 2), dtype=torch.int32, device="cuda")
    assert leg.le_bin_sort_static(cam, proj, ids, ranges) == K_ws   # warm-up: module and kernels loaded
    torch.cuda.synchronize()
    first = ids.clone()
    alloc0, free0 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
    K = leg.le_bin_sort_static(cam, proj, ids, ranges)
    torch.cuda.synchronize()
    alloc1, free1 = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
    assert K == K_ws and torch.equal(ids, first)
    assert alloc1 == alloc0
    assert free1 == free0, (free0, free1)
    del first


def test_static_scratch_limits(leg):
    import paper_2311_18482_gb300.binding as B
    # more Gaussians than the static limit: rejected before any work
    cam, proj = _project(leg, "c1", n=B_MAX_N() + 1, W=32, H=32)
    ids = torch.empty(16, dtype=torch.int32, device="cuda")
    ranges = torch.empty((4, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(B.LegError) as e:
        leg.le_bin_sort_static(cam, proj, ids, ranges)
    assert e.value.status == B.LE_ERR_INVALID_ARG
    # a capacity smaller than K: LE_ERR_CAPACITY, and K is still reported
    cam, proj = _project(leg, "c1")
    _, _, K_ws, _ = leg.le_bin_sort(cam, proj)
    ranges = torch.empty((cam.tiles_x * cam.tiles_y, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(B.LegError) as e:
        leg.le_bin_sort_static(cam, proj, ids, ranges)
    assert e.value.status == B.LE_ERR_CAPACITY
    assert e.value.k == K_ws > ids.numel()


def B_MAX_N():
    import os
    import re
    h = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "leg.h")).read()
    return int(re.search(r"#define LE_STATIC_MAX_GAUSSIANS (\d+)", h).group(1))
