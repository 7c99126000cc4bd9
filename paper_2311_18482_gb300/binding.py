"""Thin Python binding of libleg (include/leg.h).

Only argument marshalling lives here: every step of the hot path runs in the
library's CUDA kernels.  PyTorch supplies device memory and the current
stream.  If libleg.so is missing or cannot be loaded, load() raises: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libleg.so")

LE_OK, LE_ERR_INVALID_ARG, LE_ERR_CAPACITY, LE_ERR_CUDA, LE_ERR_TIMEOUT, LE_ERR_UNSUPPORTED = range(6)
UNFUSED_FP32, FUSED_BF16 = 0, 1
DECODE_TRAIN = 4          # le_decode_workspace: the workspace of a training call
SPLAT_STRIDE = 20
TILE = 16


class LegError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libleg status {status}: {msg}")
        self.status = status


class LeCamera(C.Structure):
    _fields_ = [("view", C.c_float * 12), ("campos", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("near_z", C.c_float), ("bg", C.c_float * 3)]


class LeGaussians(C.Structure):
    _fields_ = [("n", C.c_int32), ("sh_degree", C.c_int32)] + [
        (k, C.c_void_p) for k in ("means", "log_scales", "quats", "opacity_raw", "sh", "feat", "unc")]


class LeGaussianGrads(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("means", "log_scales", "quats", "opacity_raw", "sh", "feat", "unc")]


class LeAdamConfig(C.Structure):
    _fields_ = [("step", C.c_int32), ("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float)]


class LeDensifyConfig(C.Structure):
    _fields_ = [("grad_thresh", C.c_float), ("percent_dense", C.c_float), ("scene_extent", C.c_float),
                ("min_opacity", C.c_float), ("max_screen_size", C.c_float), ("world_frac", C.c_float)]


_PROJ_FIELDS = ("splat", "depth", "radius", "rect", "tiles_touched", "clamp_mask", "tile_ellipse")


class LeProjected(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in _PROJ_FIELDS]


class LeDecoder(C.Structure):
    _fields_ = [("d_in", C.c_int32), ("h1", C.c_int32), ("h2", C.c_int32), ("n_cb", C.c_int32)] + [
        (k, C.c_void_p) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]


_SMOOTH = ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")


class LeSmoothMlp(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in _SMOOTH]


class LeDecoderGrads(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]


_lib = None
_P = C.c_void_p
_SIG = {
    "le_preprocess": [C.POINTER(LeGaussians), C.POINTER(LeCamera), C.POINTER(LeProjected), _P],
    "le_bin_sort_workspace": [C.c_int32, C.c_int64, C.POINTER(C.c_size_t)],
    "le_bin_sort": [C.POINTER(LeCamera), C.c_int32, _P, _P, _P, _P, _P, C.c_size_t, C.c_int64, _P, _P, _P,
                    C.POINTER(C.c_int64), _P],
    "le_bin_sort_static": [C.POINTER(LeCamera), C.c_int32, _P, _P, _P, _P, C.c_int64, _P, _P, _P,
                           C.POINTER(C.c_int64), _P],
    "le_render_fwd": [C.POINTER(LeCamera), C.c_int32, _P, _P, _P, _P, _P, _P, _P, _P, _P],
    "le_bin_render_fwd": [C.POINTER(LeCamera), C.c_int32, _P, _P, _P, _P, _P, _P, C.c_size_t, C.c_int64, _P, _P,
                          C.POINTER(C.c_int64), _P, _P, _P, _P, _P, _P],
    "le_render_bwd": [C.POINTER(LeCamera), C.POINTER(LeGaussians), C.POINTER(LeProjected), _P, _P, _P, _P, _P, _P,
                      _P, _P, C.POINTER(LeGaussianGrads), _P],
    "le_render_bwd_adam": [C.POINTER(LeCamera), C.POINTER(LeGaussians), C.POINTER(LeProjected), _P, _P, _P, _P, _P,
                           _P, _P, _P, C.POINTER(LeGaussianGrads), C.POINTER(LeGaussianGrads),
                           C.POINTER(LeAdamConfig), _P],
    "le_render_bwd_screen": [C.POINTER(LeCamera), C.POINTER(LeGaussians), C.POINTER(LeProjected), _P, _P, _P, _P,
                             _P, _P, _P, _P, _P],
    "le_project_bwd": [C.POINTER(LeCamera), C.POINTER(LeGaussians), C.POINTER(LeProjected), _P,
                       C.POINTER(LeGaussianGrads), _P],
    "le_project_bwd_adam": [C.POINTER(LeCamera), C.POINTER(LeGaussians), C.POINTER(LeProjected), _P,
                            C.POINTER(LeGaussianGrads), C.POINTER(LeGaussianGrads), C.POINTER(LeAdamConfig), _P],
    "le_project_bwd_adam_extra": [C.POINTER(LeCamera), C.POINTER(LeGaussians), C.POINTER(LeProjected), _P,
                                  C.POINTER(LeGaussianGrads), C.POINTER(LeGaussianGrads), C.POINTER(LeAdamConfig),
                                  _P, _P, _P, _P, C.c_int64, _P],
    "le_decode_workspace": [C.c_int32, C.c_int32, C.POINTER(LeDecoder), C.POINTER(C.c_size_t)],
    "le_decode_l1": [C.c_int32, C.c_int32, _P, _P, C.POINTER(LeDecoder), _P, C.c_float, C.c_float, _P, _P, _P,
                     C.POINTER(LeDecoderGrads), _P, _P, _P, _P, _P, C.c_size_t, _P],
    "le_decode": [C.c_int32, C.c_int32, _P, _P, C.POINTER(LeDecoder), _P, C.c_float, C.c_float, _P, _P, _P,
                  C.POINTER(LeDecoderGrads), _P, _P, _P, _P, C.c_size_t, _P],
    "le_query_workspace": [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_size_t)],
    "le_query": [C.c_int32, C.c_int32, _P, C.POINTER(LeDecoder), _P, _P, C.c_int32, C.c_int32, _P, C.c_int32, _P,
                 C.c_int32, _P, _P, C.c_size_t, _P],
    "le_quantize_workspace": [C.c_int32, C.c_int32, C.POINTER(C.c_size_t)],
    "le_quantize": [C.c_int64, C.c_int32, C.c_int32, _P, C.c_int32, _P, C.c_float, C.c_float, C.c_float, _P, _P, _P,
                    _P, _P, C.c_size_t, _P],
    "le_quantize_grad_workspace": [C.c_int64, C.c_int32, C.c_int32, C.POINTER(C.c_size_t)],
    "le_quantize_grad": [C.c_int64, C.c_int32, C.c_int32, _P, C.c_int32, _P, _P, C.c_float, C.c_float, C.c_float,
                         _P, _P, C.c_size_t, _P],
    "le_smooth": [C.c_int32, _P, _P, _P, C.POINTER(LeSmoothMlp), C.c_float, C.c_float, _P, _P, C.c_int32,
                  C.POINTER(LeSmoothMlp), _P, _P],
    "le_feature_map_workspace": [C.c_int32, C.c_int32, C.POINTER(C.c_size_t)],
    "le_feature_map": [C.c_int32, _P, C.POINTER(LeDecoder), _P, C.c_int32, _P, _P, C.c_size_t, _P],
    "le_rgb_loss_workspace": [C.c_int32, C.c_int32, C.POINTER(C.c_size_t)],
    "le_rgb_loss": [C.c_int32, C.c_int32, _P, _P, C.c_float, _P, _P, _P, C.c_size_t, _P],
    "le_densify_stats": [C.c_int32, _P, _P, _P, _P, _P, _P],
    "le_opacity_reset": [C.c_int32, _P, _P, _P, C.c_float, _P],
    "le_densify_workspace": [C.c_int32, C.POINTER(C.c_size_t)],
    "le_densify": [C.POINTER(LeDensifyConfig), C.POINTER(LeGaussians), C.POINTER(LeGaussianGrads),
                   C.POINTER(LeGaussianGrads), _P, _P, _P, _P, C.c_int64, C.POINTER(LeGaussianGrads),
                   C.POINTER(LeGaussianGrads), C.POINTER(LeGaussianGrads), C.POINTER(C.c_int64), _P, C.c_size_t, _P],
    "le_rgb_l1": [C.c_int64, _P, _P, _P, _P, _P],
    "le_device_status": [_P],
    "le_selftest_bounded_wait": [_P],
    "le_adam": [C.c_int64, _P, _P, _P, _P, C.c_int32, C.c_float, C.c_float, C.c_float, C.c_float, C.c_float,
                C.c_float, _P],
}


def load():
    """Loads libleg.so (built by paper_2311_18482_gb300.build); raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} not found: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(LIB_PATH)
    for name, argtypes in _SIG.items():
        fn = getattr(lib, name, None)
        if fn is None:
            continue
        fn.argtypes = argtypes
        fn.restype = C.c_int
    lib.le_last_error.restype = C.c_char_p
    lib.le_launch_count.restype = C.c_int64
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIG) + ["le_last_error", "le_launch_count", "le_reset_launch_count"]


def _check(status: int):
    if status != LE_OK:
        raise LegError(status, load().le_last_error().decode())


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def le_device_status():
    """Synchronizes the current stream; raises LegError(LE_ERR_TIMEOUT) if a
    tensor-core kernel gave up on a bounded wait."""
    _check(load().le_device_status(_stream()))


def le_selftest_bounded_wait():
    _check(load().le_selftest_bounded_wait(_stream()))


def launch_count() -> int:
    return load().le_launch_count()


def reset_launch_count():
    load().le_reset_launch_count()


# ---------------------------------------------------------------------------
def camera_struct(cam) -> LeCamera:
    c = LeCamera()
    c.view[:] = [float(v) for v in cam.view]
    c.campos[:] = [float(v) for v in cam.campos]
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.W), int(cam.H)
    c.near_z = float(cam.near)
    c.bg[:] = [float(v) for v in cam.bg]
    return c


@dataclass
class Gaussians:
    """Device tensors of the Gaussian parameters (le_gaussians)."""
    means: torch.Tensor
    log_scales: torch.Tensor
    quats: torch.Tensor
    opacity_raw: torch.Tensor
    sh: torch.Tensor
    feat: torch.Tensor
    unc: torch.Tensor
    sh_degree: int

    @property
    def n(self) -> int:
        return self.means.shape[0]

    @staticmethod
    def from_scene(scene, device="cuda") -> "Gaussians":
        f = lambda a: torch.from_numpy(a).to(device).contiguous()
        return Gaussians(f(scene.means), f(scene.log_scales), f(scene.quats), f(scene.opacity_raw), f(scene.sh),
                         f(scene.feat), f(scene.unc), scene.sh_degree)

    def struct(self) -> LeGaussians:
        s = LeGaussians()
        s.n, s.sh_degree = self.n, self.sh_degree
        for k in ("means", "log_scales", "quats", "opacity_raw", "sh", "feat", "unc"):
            setattr(s, k, getattr(self, k).data_ptr())
        return s

    def zeros_like(self) -> "Gaussians":
        return Gaussians(*(torch.zeros_like(getattr(self, k)) for k in
                           ("means", "log_scales", "quats", "opacity_raw", "sh", "feat", "unc")), self.sh_degree)


def grads_struct(g: Gaussians) -> LeGaussianGrads:
    s = LeGaussianGrads()
    for k in ("means", "log_scales", "quats", "opacity_raw", "sh", "feat", "unc"):
        setattr(s, k, getattr(g, k).data_ptr())
    return s


@dataclass
class Projected:
    splat: torch.Tensor          # [n,20] f32
    depth: torch.Tensor          # [n] f32
    radius: torch.Tensor         # [n] i32
    rect: torch.Tensor           # [n,4] i16 (uint16 contents)
    tiles_touched: torch.Tensor  # [n] i32
    clamp_mask: torch.Tensor     # [n] u8
    tile_ellipse: torch.Tensor   # [n,8] f32

    @staticmethod
    def empty(n: int, device="cuda") -> "Projected":
        return Projected(torch.empty((n, SPLAT_STRIDE), dtype=torch.float32, device=device),
                         torch.empty(n, dtype=torch.float32, device=device),
                         torch.empty(n, dtype=torch.int32, device=device),
                         torch.empty((n, 4), dtype=torch.int16, device=device),
                         torch.empty(n, dtype=torch.int32, device=device),
                         torch.empty(n, dtype=torch.uint8, device=device),
                         torch.empty((n, 8), dtype=torch.float32, device=device))

    def struct(self) -> LeProjected:
        s = LeProjected()
        for k in _PROJ_FIELDS:
            setattr(s, k, getattr(self, k).data_ptr())
        return s


# ---------------------------------------------------------------------------
# Entry points (same names as the C ABI)

def le_preprocess(g: Gaussians, cam, out: Projected | None = None) -> Projected:
    out = out or Projected.empty(g.n, g.means.device)
    gs, cs, ps = g.struct(), camera_struct(cam), out.struct()
    _check(load().le_preprocess(C.byref(gs), C.byref(cs), C.byref(ps), _stream()))
    return out


def le_bin_sort_workspace(n: int, k_cap: int) -> int:
    b = C.c_size_t()
    _check(load().le_bin_sort_workspace(n, k_cap, C.byref(b)))
    return b.value


class BinSortBuffers:
    """Reusable device buffers for le_bin_sort (grown on demand)."""

    def __init__(self):
        self.ws = None
        self.ids = None
        self.keys = None
        self.ranges = None
        self.n = self.k_cap = -1

    def ensure(self, n, k_cap, ntiles, device, want_keys=False):
        if self.ws is None or n > self.n or k_cap > self.k_cap:
            self.n, self.k_cap = max(n, self.n), max(k_cap, self.k_cap)
            nb = le_bin_sort_workspace(self.n, self.k_cap)
            self.ws = torch.empty(nb, dtype=torch.uint8, device=device)
            self.ids = torch.empty(max(self.k_cap, 1), dtype=torch.int32, device=device)
            self.keys = None
        if want_keys and (self.keys is None or self.keys.numel() < self.k_cap):
            self.keys = torch.empty(max(self.k_cap, 1), dtype=torch.int64, device=device)
        if self.ranges is None or self.ranges.shape[0] < ntiles:
            self.ranges = torch.empty((ntiles, 2), dtype=torch.int32, device=device)


def le_bin_sort(cam, proj: Projected, buffers: BinSortBuffers | None = None, k_cap: int | None = None,
                want_keys: bool = False):
    """Returns (sorted_ids[K] int32 (uint32 contents), tile_ranges[T,2], K, sorted_keys or None).
    Retries once with a larger capacity on LE_ERR_CAPACITY."""
    n = proj.depth.shape[0]
    ntiles = ((cam.W + TILE - 1) // TILE) * ((cam.H + TILE - 1) // TILE)
    buffers = buffers or BinSortBuffers()
    k_cap = k_cap if k_cap is not None else max(buffers.k_cap, 16 * n, 1024)
    cs = camera_struct(cam)
    for _ in range(2):
        buffers.ensure(n, k_cap, ntiles, proj.depth.device, want_keys)
        K = C.c_int64()
        st = load().le_bin_sort(C.byref(cs), n, _ptr(proj.depth), _ptr(proj.rect), _ptr(proj.tile_ellipse),
                                _ptr(proj.tiles_touched), _ptr(buffers.ws), buffers.ws.numel(), buffers.k_cap, _ptr(buffers.ids),
                                _ptr(buffers.keys) if want_keys else None, _ptr(buffers.ranges), C.byref(K),
                                _stream())
        if st == LE_ERR_CAPACITY:
            k_cap = int(K.value * 1.25) + 1024
            continue
        _check(st)
        k = K.value
        return (buffers.ids[:k], buffers.ranges[:ntiles], k,
                buffers.keys[:k] if want_keys else None)
    raise LegError(LE_ERR_CAPACITY, "capacity retry failed")


def le_bin_sort_static(cam, proj: Projected, sorted_ids, tile_ranges, sorted_keys=None):
    """le_bin_sort with the library's static scratch (no workspace; see leg.h).
    The caller provides the outputs; returns K.  On LE_ERR_CAPACITY the raised
    LegError carries the instance count the call reported as `.k`."""
    K = C.c_int64()
    st = load().le_bin_sort_static(C.byref(camera_struct(cam)), proj.depth.shape[0], _ptr(proj.depth),
                                   _ptr(proj.rect), _ptr(proj.tile_ellipse), _ptr(proj.tiles_touched),
                                   sorted_ids.numel(),
                                   _ptr(sorted_ids), _ptr(sorted_keys), _ptr(tile_ranges), C.byref(K), _stream())
    if st != LE_OK:
        err = LegError(st, load().le_last_error().decode())
        err.k = K.value
        raise err
    return K.value


@dataclass
class Image:
    rgb: torch.Tensor       # [3,H,W]
    feat: torch.Tensor      # [8,H,W]
    unc: torch.Tensor       # [H,W]
    T: torch.Tensor         # [H,W]
    n_contrib: torch.Tensor  # [H,W] i32

    @staticmethod
    def empty(H, W, device="cuda"):
        f = lambda *s: torch.empty(s, dtype=torch.float32, device=device)
        return Image(f(3, H, W), f(8, H, W), f(H, W), f(H, W), torch.empty((H, W), dtype=torch.int32, device=device))


def le_render_fwd(cam, proj: Projected, ids, ranges, out: Image | None = None) -> Image:
    out = out or Image.empty(cam.H, cam.W, proj.splat.device)
    cs = camera_struct(cam)
    _check(load().le_render_fwd(C.byref(cs), proj.splat.shape[0], _ptr(proj.splat), _ptr(ids), _ptr(ranges),
                                _ptr(out.rgb), _ptr(out.feat), _ptr(out.unc), _ptr(out.T), _ptr(out.n_contrib),
                                _stream()))
    return out


def le_bin_render_fwd(cam, proj: Projected, buffers: BinSortBuffers | None = None, out: Image | None = None,
                      k_cap: int | None = None):
    """le_bin_sort + le_render_fwd with lazy placement (see leg.h).  Returns
    (sorted_ids, tile_ranges, K, image); ids are written up to every tile's
    last reached entry.  Retries once with a larger capacity on LE_ERR_CAPACITY."""
    n = proj.depth.shape[0]
    ntiles = ((cam.W + TILE - 1) // TILE) * ((cam.H + TILE - 1) // TILE)
    buffers = buffers or BinSortBuffers()
    out = out or Image.empty(cam.H, cam.W, proj.splat.device)
    k_cap = k_cap if k_cap is not None else max(buffers.k_cap, 16 * n, 1024)
    cs = camera_struct(cam)
    for _ in range(2):
        buffers.ensure(n, k_cap, ntiles, proj.depth.device)
        K = C.c_int64()
        st = load().le_bin_render_fwd(C.byref(cs), n, _ptr(proj.splat), _ptr(proj.depth), _ptr(proj.rect),
                                      _ptr(proj.tile_ellipse), _ptr(proj.tiles_touched), _ptr(buffers.ws),
                                      buffers.ws.numel(), buffers.k_cap, _ptr(buffers.ids), _ptr(buffers.ranges),
                                      C.byref(K), _ptr(out.rgb), _ptr(out.feat), _ptr(out.unc), _ptr(out.T),
                                      _ptr(out.n_contrib), _stream())
        if st == LE_ERR_CAPACITY:
            k_cap = int(K.value * 1.25) + 1024
            continue
        _check(st)
        k = K.value
        return buffers.ids[:k], buffers.ranges[:ntiles], k, out
    raise LegError(LE_ERR_CAPACITY, "capacity retry failed")


def le_render_bwd(cam, g: Gaussians, proj: Projected, ids, ranges, img: Image, dL_drgb, dL_dfeat, dL_dunc,
                  grads: Gaussians | None = None, grad2d=None):
    grads = grads or g.zeros_like()
    grad2d = grad2d if grad2d is not None else torch.empty((g.n, SPLAT_STRIDE), dtype=torch.float32,
                                                           device=g.means.device)
    cs, gs, ps, os_ = camera_struct(cam), g.struct(), proj.struct(), grads_struct(grads)
    _check(load().le_render_bwd(C.byref(cs), C.byref(gs), C.byref(ps), _ptr(ids), _ptr(ranges), _ptr(img.T),
                                _ptr(img.n_contrib), _ptr(dL_drgb.contiguous()), _ptr(dL_dfeat.contiguous()),
                                _ptr(dL_dunc.contiguous()), _ptr(grad2d), C.byref(os_), _stream()))
    return grads, grad2d


def le_render_bwd_adam(cam, g: Gaussians, proj: Projected, ids, ranges, img: Image, dL_drgb, dL_dfeat, dL_dunc,
                       m: Gaussians, v: Gaussians, step: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                       grad2d=None):
    """le_render_bwd with the Adam step fused in: updates g's tensors (and m, v) in place."""
    grad2d = grad2d if grad2d is not None else torch.empty((g.n, SPLAT_STRIDE), dtype=torch.float32,
                                                           device=g.means.device)
    cs, gs, ps = camera_struct(cam), g.struct(), proj.struct()
    ms, vs = grads_struct(m), grads_struct(v)
    cfg = LeAdamConfig(int(step), lr, beta1, beta2, eps)
    _check(load().le_render_bwd_adam(C.byref(cs), C.byref(gs), C.byref(ps), _ptr(ids), _ptr(ranges), _ptr(img.T),
                                     _ptr(img.n_contrib), _ptr(dL_drgb.contiguous()), _ptr(dL_dfeat.contiguous()),
                                     _ptr(dL_dunc.contiguous()), _ptr(grad2d), C.byref(ms), C.byref(vs),
                                     C.byref(cfg), _stream()))
    return grad2d


def le_render_bwd_screen(cam, g: Gaussians, proj: Projected, ids, ranges, img: Image, dL_drgb, dL_dfeat, dL_dunc,
                         grad2d=None):
    """Screen-space half of le_render_bwd: returns grad2d [n, 20]."""
    grad2d = grad2d if grad2d is not None else torch.empty((g.n, SPLAT_STRIDE), dtype=torch.float32,
                                                           device=g.means.device)
    cs, gs, ps = camera_struct(cam), g.struct(), proj.struct()
    _check(load().le_render_bwd_screen(C.byref(cs), C.byref(gs), C.byref(ps), _ptr(ids), _ptr(ranges), _ptr(img.T),
                                       _ptr(img.n_contrib), _ptr(dL_drgb.contiguous()), _ptr(dL_dfeat.contiguous()),
                                       _ptr(dL_dunc.contiguous()), _ptr(grad2d), _stream()))
    return grad2d


def le_project_bwd(cam, g: Gaussians, proj: Projected, grad2d, grads: Gaussians | None = None) -> Gaussians:
    """Projection half of le_render_bwd: parameter gradients from grad2d."""
    grads = grads or g.zeros_like()
    cs, gs, ps, os_ = camera_struct(cam), g.struct(), proj.struct(), grads_struct(grads)
    _check(load().le_project_bwd(C.byref(cs), C.byref(gs), C.byref(ps), _ptr(grad2d), C.byref(os_), _stream()))
    return grads


def le_project_bwd_adam(cam, g: Gaussians, proj: Projected, grad2d, m: Gaussians, v: Gaussians, step: int, lr=1e-3,
                        beta1=0.9, beta2=0.999, eps=1e-8):
    """Projection half of le_render_bwd_adam: the Adam step on g's tensors (and m, v) in place."""
    cs, gs, ps = camera_struct(cam), g.struct(), proj.struct()
    ms, vs = grads_struct(m), grads_struct(v)
    cfg = LeAdamConfig(int(step), lr, beta1, beta2, eps)
    _check(load().le_project_bwd_adam(C.byref(cs), C.byref(gs), C.byref(ps), _ptr(grad2d), C.byref(ms),
                                      C.byref(vs), C.byref(cfg), _stream()))


def le_project_bwd_adam_extra(cam, g: Gaussians, proj: Projected, grad2d, m: Gaussians, v: Gaussians, step: int,
                              extra_param, extra_grad, extra_m, extra_v, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """le_project_bwd_adam plus the same Adam step on one more flat FP32 range (extra_*, equal sizes)."""
    n = extra_param.numel()
    assert extra_grad.numel() == n and extra_m.numel() == n and extra_v.numel() == n
    cs, gs, ps = camera_struct(cam), g.struct(), proj.struct()
    ms, vs = grads_struct(m), grads_struct(v)
    cfg = LeAdamConfig(int(step), lr, beta1, beta2, eps)
    _check(load().le_project_bwd_adam_extra(C.byref(cs), C.byref(gs), C.byref(ps), _ptr(grad2d), C.byref(ms),
                                            C.byref(vs), C.byref(cfg), _ptr(extra_param), _ptr(extra_grad),
                                            _ptr(extra_m), _ptr(extra_v), C.c_int64(n), _stream()))


def decoder_struct(W1, b1, W2, b2, W3, b3) -> LeDecoder:
    d = LeDecoder()
    d.d_in, d.h1, d.h2, d.n_cb = W1.shape[1], W1.shape[0], W2.shape[0], W3.shape[0]
    d.W1, d.b1, d.W2, d.b2, d.W3, d.b3 = (t.data_ptr() for t in (W1, b1, W2, b2, W3, b3))
    return d


def le_decode_workspace(mode: int, P: int, dec: LeDecoder) -> int:
    b = C.c_size_t()
    _check(load().le_decode_workspace(mode, P, C.byref(dec), C.byref(b)))
    return b.value


def decoder_grads_struct(dW) -> LeDecoderGrads:
    dg = LeDecoderGrads()
    dg.W1, dg.b1, dg.W2, dg.b2, dg.W3, dg.b3 = (t.data_ptr() for t in dW)
    return dg


def le_decode_raw(mode, P, feat, unc, dec: LeDecoder, target, lambda_ce, lambda_u, loss, d_feat, d_unc,
                  dgrads: LeDecoderGrads | None, argmax, prob, logits, workspace):
    """Direct call with preallocated device tensors (any of the outputs may be None)."""
    _check(load().le_decode(mode, P, _ptr(feat), _ptr(unc), C.byref(dec), _ptr(target), lambda_ce, lambda_u,
                            _ptr(loss), _ptr(d_feat), _ptr(d_unc), C.byref(dgrads) if dgrads is not None else None,
                            _ptr(argmax), _ptr(prob), _ptr(logits), _ptr(workspace),
                            0 if workspace is None else workspace.numel(), _stream()))


def le_decode_l1_raw(mode, P, feat, unc, dec: LeDecoder, target, lambda_ce, lambda_u, loss, d_feat, d_unc,
                     dgrads: LeDecoderGrads, img, img_target, loss_l1, d_img, workspace):
    """A training call of le_decode plus the RGB L1 term of the same pixels (preallocated tensors)."""
    _check(load().le_decode_l1(mode, P, _ptr(feat), _ptr(unc), C.byref(dec), _ptr(target), lambda_ce, lambda_u,
                               _ptr(loss), _ptr(d_feat), _ptr(d_unc), C.byref(dgrads), _ptr(img), _ptr(img_target),
                               _ptr(loss_l1), _ptr(d_img), _ptr(workspace),
                               0 if workspace is None else workspace.numel(), _stream()))


def le_decode(mode: int, feat, dec_t, unc=None, target=None, lambda_ce=1.0, lambda_u=1.0, want_prob=False,
              want_logits=False, want_argmax=True, workspace=None):
    """dec_t = (W1, b1, W2, b2, W3, b3) device tensors.  Allocates outputs; returns a dict."""
    P = feat.shape[-1] * (feat.shape[-2] if feat.dim() == 3 else 1)
    dev = feat.device
    dec = decoder_struct(*dec_t)
    ncb = dec.n_cb
    nb = le_decode_workspace(mode | (DECODE_TRAIN if target is not None else 0), P, dec)
    if workspace is None or workspace.numel() < nb:
        workspace = torch.empty(max(nb, 1), dtype=torch.uint8, device=dev)
    out = {}
    train = target is not None
    dg = None
    if train:
        out["loss"] = torch.zeros(2, dtype=torch.float32, device=dev)
        out["d_feat"] = torch.empty((8, P), dtype=torch.float32, device=dev)
        out["d_unc"] = torch.empty(P, dtype=torch.float32, device=dev)
        out["dW"] = [torch.empty_like(t) for t in dec_t]
        dg = decoder_grads_struct(out["dW"])
    if want_argmax:
        out["argmax"] = torch.empty(P, dtype=torch.int32, device=dev)
    if want_prob:
        out["prob"] = torch.empty((ncb, P), dtype=torch.float32, device=dev)
    if want_logits:
        out["logits"] = torch.empty((ncb, P), dtype=torch.float32, device=dev)
    le_decode_raw(mode, P, feat.contiguous(), unc.contiguous() if unc is not None else None, dec,
                  target.contiguous() if train else None, lambda_ce, lambda_u, out.get("loss"), out.get("d_feat"),
                  out.get("d_unc"), dg, out.get("argmax"), out.get("prob"), out.get("logits"), workspace)
    out["workspace"] = workspace
    return out


def le_query_workspace(mode: int, P: int, n_cb: int, d_clip: int) -> int:
    b = C.c_size_t()
    _check(load().le_query_workspace(mode, P, n_cb, d_clip, C.byref(b)))
    return b.value


def le_query(mode: int, P: int, codebook, d_clip: int, text, negs, feat=None, dec_t=None, prob=None,
             workspace=None, out=None):
    dev = codebook.device
    n_cb, d = codebook.shape
    nb = le_query_workspace(mode, P, n_cb, d_clip)
    if workspace is None or workspace.numel() < nb:
        workspace = torch.empty(max(nb, 1), dtype=torch.uint8, device=dev)
    Q = text.shape[0]
    out = out if out is not None else torch.empty((Q, P), dtype=torch.float32, device=dev)
    dec = decoder_struct(*dec_t) if dec_t is not None else None
    _check(load().le_query(mode, P, _ptr(feat), C.byref(dec) if dec is not None else None, _ptr(prob),
                           _ptr(codebook), d, d_clip, _ptr(text), Q, _ptr(negs), negs.shape[0], _ptr(out),
                           _ptr(workspace), workspace.numel(), _stream()))
    return out


def le_quantize_workspace(n_cb: int, d: int) -> int:
    n = C.c_size_t()
    _check(load().le_quantize_workspace(n_cb, d, C.byref(n)))
    return n.value


def le_quantize(features, codebook, d_clip=512, lambda_d=0.5, lambda_cos=1.0, lambda_lb=0.5, out=None,
                workspace=None):
    """Quantisation of language features (Sec. 3.3): features [K, d] torch.bfloat16 (or int16
    holding BF16 bits), codebook [N, d] float32.  Returns (indices [K] int32, r [N], p [N],
    loss [3] = (L_q, L_cos, L_lb)), all device tensors."""
    K, d = features.shape
    N = codebook.shape[0]
    dev = features.device
    if out is None:
        out = (torch.empty(K, dtype=torch.int32, device=dev), torch.empty(N, dtype=torch.float32, device=dev),
               torch.empty(N, dtype=torch.float32, device=dev), torch.empty(3, dtype=torch.float32, device=dev))
    idx, r, p, loss = out
    if workspace is None:
        workspace = torch.empty(max(le_quantize_workspace(N, d), 1), dtype=torch.uint8, device=dev)
    _check(load().le_quantize(K, d, d_clip, _ptr(features), N, _ptr(codebook.contiguous()), lambda_d, lambda_cos,
                              lambda_lb, _ptr(idx), _ptr(r), _ptr(p), _ptr(loss), _ptr(workspace), workspace.numel(),
                              _stream()))
    return idx, r, p, loss


def le_quantize_grad_workspace(K: int, n_cb: int, d: int) -> int:
    n = C.c_size_t()
    _check(load().le_quantize_grad_workspace(K, n_cb, d, C.byref(n)))
    return n.value


def le_quantize_grad(features, codebook, r, d_clip=512, lambda_d=0.5, lambda_cos=1.0, lambda_lb=0.5, out=None,
                     workspace=None):
    """Gradient of L_q with respect to the codebook (Sec. 3.3): features [K, d] BF16 (or int16
    bits), codebook [N, d] float32, r [N] from le_quantize.  Returns grad [N, d] float32."""
    K, d = features.shape
    N = codebook.shape[0]
    dev = features.device
    out = out if out is not None else torch.empty((N, d), dtype=torch.float32, device=dev)
    if workspace is None:
        workspace = torch.empty(le_quantize_grad_workspace(K, N, d), dtype=torch.uint8, device=dev)
    _check(load().le_quantize_grad(K, d, d_clip, _ptr(features), N, _ptr(codebook.contiguous()), _ptr(r), lambda_d,
                                   lambda_cos, lambda_lb, _ptr(out), _ptr(workspace), workspace.numel(), _stream()))
    return out


def smooth_struct(params) -> LeSmoothMlp:
    """params: sequence or dict of the 8 MLP tensors (W1, b1, ..., W4, b4), contiguous FP32."""
    s = LeSmoothMlp()
    vals = [params[k] for k in _SMOOTH] if isinstance(params, dict) else list(params)
    for k, t in zip(_SMOOTH, vals):
        setattr(s, k, t.data_ptr())
    return s


def le_smooth(means, feat, unc, mlp, w_s=0.1, lambda_smo=1.0, d_feat=None, d_feat_stride=8, grads=None,
              want_s_mlp=False):
    """Adaptive spatial smoothing (Sec. 3.4): returns (loss [1], d_feat, grads list, s_mlp or None).
    d_feat is ADDED to (a zeroed [n, 8] array when not given)."""
    n = means.shape[0]
    dev = means.device
    vals = [mlp[k] for k in _SMOOTH] if isinstance(mlp, dict) else list(mlp)
    if d_feat is None:
        d_feat = torch.zeros((n, 8), dtype=torch.float32, device=dev)
    if grads is None:
        grads = [torch.empty_like(v) for v in vals]
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    s_mlp = torch.empty((n, 8), dtype=torch.float32, device=dev) if want_s_mlp else None
    ms, gs = smooth_struct(vals), smooth_struct(grads)
    _check(load().le_smooth(n, _ptr(means), _ptr(feat), _ptr(unc), C.byref(ms), w_s, lambda_smo, _ptr(loss),
                            _ptr(d_feat), d_feat_stride, C.byref(gs), _ptr(s_mlp), _stream()))
    return loss, d_feat, grads, s_mlp


def le_feature_map(feat, dec_t, codebook, out=None, workspace=None):
    """F = softmax(D_MLP(feat)) S (supp. Sec. "Inference"): feat [8, P], dec_t the six decoder tensors,
    codebook [N, d] float32.  Returns F [P, d] as torch.bfloat16."""
    P = feat.shape[1]
    N, d = codebook.shape
    dev = feat.device
    out = out if out is not None else torch.empty((P, d), dtype=torch.bfloat16, device=dev)
    dec = decoder_struct(*dec_t)
    if workspace is None:
        n = C.c_size_t()
        _check(load().le_feature_map_workspace(N, d, C.byref(n)))
        workspace = torch.empty(n.value, dtype=torch.uint8, device=dev)
    _check(load().le_feature_map(P, _ptr(feat.contiguous()), C.byref(dec), _ptr(codebook.contiguous()), d, _ptr(out),
                                 _ptr(workspace), workspace.numel(), _stream()))
    return out


def le_rgb_loss_workspace(W: int, H: int) -> int:
    n = C.c_size_t()
    _check(load().le_rgb_loss_workspace(W, H, C.byref(n)))
    return n.value


def le_rgb_loss(img, target, lambda_ssim=0.2, loss=None, grad=None, workspace=None):
    """(1 - lambda) L1 + lambda (1 - SSIM) on [3, H, W] images: returns (loss [3] = (L, L1, SSIM), grad)."""
    _, H, W = img.shape
    dev = img.device
    loss = loss if loss is not None else torch.empty(3, dtype=torch.float32, device=dev)
    grad = grad if grad is not None else torch.empty_like(img)
    if workspace is None:
        workspace = torch.empty(le_rgb_loss_workspace(W, H), dtype=torch.uint8, device=dev)
    _check(load().le_rgb_loss(W, H, _ptr(img.contiguous()), _ptr(target.contiguous()), lambda_ssim, _ptr(loss),
                              _ptr(grad), _ptr(workspace), workspace.numel(), _stream()))
    return loss, grad


def le_densify_stats(grad2d, radius, acc, cnt, max_radius=None):
    """acc [n] float32 += |dL/dmean2d|, cnt [n] int32 += 1 and max_radius [n] int32 (optional)
    = max(max_radius, radius) for every visible Gaussian (in place)."""
    _check(load().le_densify_stats(acc.shape[0], _ptr(grad2d), _ptr(radius), _ptr(acc), _ptr(cnt),
                                   _ptr(max_radius), _stream()))


def le_opacity_reset(opacity_raw, m_opacity, v_opacity, max_opacity=0.01):
    """In place: opacity = min(opacity, max_opacity) and the opacity's Adam moments zeroed."""
    _check(load().le_opacity_reset(opacity_raw.numel(), _ptr(opacity_raw), _ptr(m_opacity), _ptr(v_opacity),
                                   max_opacity, _stream()))


def le_densify(g: Gaussians, m: Gaussians, v: Gaussians, acc, cnt, noise, grad_thresh=0.0002, percent_dense=0.01,
               scene_extent=1.0, min_opacity=0.005, n_cap=None, max_radius=None, max_screen_size=0.0,
               world_frac=0.0):
    """Adaptive density control: returns (g', m', v') as Gaussians of the new size.  max_screen_size
    (pixels, needs max_radius) and world_frac (of scene_extent) > 0 turn on the size pruning."""
    n = g.n
    n_cap = n_cap if n_cap is not None else 2 * n
    grow = lambda t: torch.empty((n_cap,) + tuple(t.shape[1:]), dtype=t.dtype, device=t.device)
    outs = [Gaussians(*(grow(getattr(x, k)) for k in ("means", "log_scales", "quats", "opacity_raw", "sh", "feat",
                                                       "unc")), g.sh_degree) for x in (g, g, g)]
    cfg = LeDensifyConfig(grad_thresh, percent_dense, scene_extent, min_opacity, max_screen_size, world_frac)
    ws_n = C.c_size_t()
    _check(load().le_densify_workspace(n, C.byref(ws_n)))
    ws = torch.empty(max(ws_n.value, 1), dtype=torch.uint8, device=g.means.device)
    n_out = C.c_int64()
    gs, ms, vs = g.struct(), grads_struct(m), grads_struct(v)
    os_ = [grads_struct(o) for o in outs]
    _check(load().le_densify(C.byref(cfg), C.byref(gs), C.byref(ms), C.byref(vs), _ptr(acc), _ptr(cnt),
                             _ptr(max_radius), _ptr(noise.contiguous()), n_cap, C.byref(os_[0]), C.byref(os_[1]), C.byref(os_[2]),
                             C.byref(n_out), _ptr(ws), ws.numel(), _stream()))
    k = n_out.value
    cut = lambda o: Gaussians(*(getattr(o, f)[:k] for f in ("means", "log_scales", "quats", "opacity_raw", "sh",
                                                          "feat", "unc")), o.sh_degree)
    return cut(outs[0]), cut(outs[1]), cut(outs[2])


def le_rgb_l1(img, target, loss, grad):
    _check(load().le_rgb_l1(img.numel(), _ptr(img), _ptr(target), _ptr(loss), _ptr(grad), _stream()))


def le_adam(param, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, clamp_lo=-float("inf"),
            clamp_hi=float("inf")):
    _check(load().le_adam(param.numel(), _ptr(param), _ptr(grad), _ptr(m), _ptr(v), int(step), lr, beta1, beta2,
                          eps, clamp_lo, clamp_hi, _stream()))


# ---------------------------------------------------------------------------
_K_HINT = {}   # device -> the last rasterize call's instance count K


class _Rasterize(torch.autograd.Function):
    """Differentiable rasterization (Eq. 1 plus R_s and R_u): returns
    (rgb [3,H,W], feat [8,H,W], unc [H,W]); backward returns gradients for
    means, log_scales, quats, opacity_raw, sh, feat, unc.  The forward bins and
    renders with lazily placed lists (le_bin_render_fwd: the entries any pixel
    reads, which is all the backward reads)."""

    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_raw, sh, feat, unc, cam, sh_degree, buffers):
        g = Gaussians(means.contiguous(), log_scales.contiguous(), quats.contiguous(), opacity_raw.contiguous(),
                      sh.contiguous(), feat.contiguous(), unc.contiguous(), sh_degree)
        proj = le_preprocess(g, cam)
        own = buffers is None
        # fresh lists sized from the previous call's K on this device (one binning, no capacity retry)
        hint = _K_HINT.get(means.device)
        k_cap = max(16 * g.n, int(1.25 * hint) + 1024) if own and hint is not None else None
        ids, ranges, K, img = le_bin_render_fwd(cam, proj, BinSortBuffers() if own else buffers, k_cap=k_cap)
        _K_HINT[means.device] = K
        # buffers the caller reuses may be overwritten by a later forward before this backward
        ctx.cam, ctx.g, ctx.proj, ctx.img = cam, g, proj, img
        ctx.ids, ctx.ranges = (ids, ranges) if own else (ids.clone(), ranges.clone())
        ctx.mark_non_differentiable(img.T)
        return img.rgb, img.feat, img.unc, img.T

    @staticmethod
    def backward(ctx, d_rgb, d_feat, d_unc, d_T):
        H, W = ctx.cam.H, ctx.cam.W
        dev = ctx.g.means.device
        z = lambda *s: torch.zeros(s, dtype=torch.float32, device=dev)
        d_rgb = d_rgb if d_rgb is not None else z(3, H, W)
        d_feat = d_feat if d_feat is not None else z(8, H, W)
        d_unc = d_unc if d_unc is not None else z(H, W)
        grads, _ = le_render_bwd(ctx.cam, ctx.g, ctx.proj, ctx.ids, ctx.ranges, ctx.img, d_rgb, d_feat, d_unc)
        return (grads.means, grads.log_scales, grads.quats, grads.opacity_raw, grads.sh, grads.feat, grads.unc,
                None, None, None)


def rasterize(means, log_scales, quats, opacity_raw, sh, feat, unc, cam, sh_degree, buffers=None):
    """Autograd entry: (rgb, feat, unc, T_final) images of the Gaussians seen from `cam`.  buffers
    (optional): BinSortBuffers reused across calls (the lists are then copied for the backward)."""
    return _Rasterize.apply(means, log_scales, quats, opacity_raw, sh, feat, unc, cam, sh_degree, buffers)
