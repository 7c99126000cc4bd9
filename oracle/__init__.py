"""FP64 CPU oracle for the Language Embedded 3D Gaussians hot path.

TEST INFRASTRUCTURE ONLY: imported by `tests/`, `__graft_entry__.smoke()` and
the CPU-baseline leg of `bench.py`, never by the product package.  It shares
no code with the CUDA library.  The C sources in this directory state what
each step computes and which passage of the paper it follows; this module
only compiles them (gcc, -ffp-contract=off) and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sysconfig

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["keypath.c", "sh.c", "project.c", "binning.c", "composite.c", "decoder.c", "query.c", "train.c",
           "quant.c", "smooth.c", "ssim.c", "densify.c"]
LIB = os.path.join(HERE, "liboracle.so")
TILE = 16


def build(force: bool = False) -> str:
    """Compile liboracle.so in place (plain C11, FP64, OpenMP over pixels)."""
    srcs = [os.path.join(HERE, s) for s in SOURCES]
    if not force and os.path.exists(LIB):
        newest = max(os.path.getmtime(p) for p in srcs + [os.path.join(HERE, "oracle.h")])
        if os.path.getmtime(LIB) >= newest:
            return LIB
    cmd = ["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-Wall", "-Wno-unused-function", "-o", LIB + ".tmp"] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(LIB)
        _lib.orc_exp_f32.restype = C.c_float
        _lib.orc_exp_f32.argtypes = [C.c_float]
        _lib.orc_ln_up_f32.restype = C.c_float
        _lib.orc_ln_up_f32.argtypes = [C.c_float]
        _lib.orc_bin.restype = C.c_int64
        _lib.orc_bin_count.restype = C.c_int64
        _lib.orc_tile_list.restype = C.c_int
        _lib.orc_l1.restype = C.c_double
        _lib.orc_sh_count.restype = C.c_int
        _lib.orc_densify_plan.restype = C.c_int64
        _lib.orc_bf16_bits.restype = C.c_uint16
        _lib.orc_bf16_bits.argtypes = [C.c_float]
    return _lib


class OrcCam(C.Structure):
    _fields_ = [("view", C.c_float * 12), ("campos", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("W", C.c_int32), ("H", C.c_int32),
                ("near_z", C.c_float), ("bg", C.c_float * 3)]


def cam_struct(cam) -> OrcCam:
    c = OrcCam()
    c.view[:] = [float(v) for v in np.asarray(cam.view, np.float32)]
    c.campos[:] = [float(v) for v in np.asarray(cam.campos, np.float32)]
    c.fx, c.fy, c.cx, c.cy = cam.fx, cam.fy, cam.cx, cam.cy
    c.W, c.H = cam.W, cam.H
    c.near_z = cam.near
    c.bg[:] = [float(v) for v in np.asarray(cam.bg, np.float32)]
    return c


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, np.float32)


def _f64(a):
    return np.ascontiguousarray(a, np.float64)


def exp_f32(x: float) -> float:
    return lib().orc_exp_f32(float(x))


def ln_up_f32(x: float) -> float:
    return lib().orc_ln_up_f32(float(x))


def sh_basis(deg: int, d):
    n = (deg + 1) ** 2
    d = _f64(d)
    Y = np.zeros(n)
    dY = np.zeros((n, 3))
    lib().orc_sh_basis(C.c_int(deg), _p(d), _p(Y), _p(dY))
    return Y, dY


def keypath(scene, cam) -> dict:
    N = scene.N
    out = dict(depth=np.zeros(N, np.float32), mean2d=np.zeros((N, 2), np.float32),
               cov2d=np.zeros((N, 3), np.float32), radius=np.zeros(N, np.int32),
               rect=np.zeros((N, 4), np.int32), tiles=np.zeros(N, np.int32), ell=np.zeros((N, 8), np.float32))
    cs = cam_struct(cam)
    m, ls, q, o = _f32(scene.means), _f32(scene.log_scales), _f32(scene.quats), _f32(scene.opacity_raw)
    lib().orc_keypath(C.c_int(N), _p(m), _p(ls), _p(q), _p(o), C.byref(cs), _p(out["depth"]), _p(out["mean2d"]),
                      _p(out["cov2d"]), _p(out["radius"]), _p(out["rect"]), _p(out["tiles"]), _p(out["ell"]))
    return out


def row_span(kp, i: int, ty: int):
    """Tiles [xl, xr) of row ty of Gaussian i's rectangle that meet its tile ellipse."""
    xl, xr = C.c_int(), C.c_int()
    e = np.ascontiguousarray(kp["ell"][i], np.float32)
    r = np.ascontiguousarray(kp["rect"][i], np.int32)
    lib().orc_row_span(_p(e), _p(r), C.c_int(ty), C.byref(xl), C.byref(xr))
    return xl.value, xr.value


def project(scene, cam, tiles) -> dict:
    N = scene.N
    out = dict(mean2d=np.zeros((N, 2)), depth=np.zeros(N), cov2d=np.zeros((N, 3)), conic=np.zeros((N, 3)),
               opacity=np.zeros(N), rgb=np.zeros((N, 3)), clamp=np.zeros(N, np.uint8))
    cs = cam_struct(cam)
    args = [_f64(scene.means), _f64(scene.log_scales), _f64(scene.quats), _f64(scene.opacity_raw), _f64(scene.sh)]
    tiles = np.ascontiguousarray(tiles, np.int32)
    lib().orc_project(C.c_int(N), C.c_int(scene.sh_degree), *[_p(a) for a in args], C.byref(cs), _p(tiles),
                      _p(out["mean2d"]), _p(out["depth"]), _p(out["cov2d"]), _p(out["conic"]),
                      _p(out["opacity"]), _p(out["rgb"]), _p(out["clamp"]))
    return out


def project_bwd(scene, cam, tiles, d_mean2d, d_conic, d_opacity, d_rgb) -> dict:
    N = scene.N
    nc = (scene.sh_degree + 1) ** 2
    out = dict(means=np.zeros((N, 3)), log_scales=np.zeros((N, 3)), quats=np.zeros((N, 4)),
               opacity_raw=np.zeros(N), sh=np.zeros((N, nc, 3)))
    cs = cam_struct(cam)
    args = [_f64(scene.means), _f64(scene.log_scales), _f64(scene.quats), _f64(scene.opacity_raw), _f64(scene.sh)]
    tiles = np.ascontiguousarray(tiles, np.int32)
    g = [_f64(d_mean2d), _f64(d_conic), _f64(d_opacity), _f64(d_rgb)]
    lib().orc_project_bwd(C.c_int(N), C.c_int(scene.sh_degree), *[_p(a) for a in args], C.byref(cs), _p(tiles),
                          *[_p(a) for a in g], _p(out["means"]), _p(out["log_scales"]), _p(out["quats"]),
                          _p(out["opacity_raw"]), _p(out["sh"]))
    return out


def _ell(kp, ellipse: bool):
    return _p(kp["ell"]) if ellipse else None


def bin(cam, kp, ellipse: bool = True):
    """Keys, sorted Gaussian ids and per-tile ranges (stable sort of 64-bit keys).
    ellipse=False bins whole rectangles (the plain 3DGS assignment)."""
    N = kp["tiles"].shape[0]
    cap = int(kp["tiles"].astype(np.int64).sum())
    keys = np.zeros(max(cap, 1), np.uint64)
    vals = np.zeros(max(cap, 1), np.uint32)
    ntiles = cam.tiles_x * cam.tiles_y
    ranges = np.zeros((ntiles, 2), np.uint32)
    cs = cam_struct(cam)
    K = lib().orc_bin(C.c_int(N), C.byref(cs), _p(kp["depth"]), _p(kp["rect"]), _p(kp["tiles"]),
                      _ell(kp, ellipse), _p(keys), _p(vals), _p(ranges))
    assert 0 <= K <= cap
    return keys[:K], vals[:K], ranges


def bin_count(kp, ellipse: bool = True) -> int:
    """The number of tile copies bin() emits."""
    N = kp["tiles"].shape[0]
    return int(lib().orc_bin_count(C.c_int(N), _p(kp["rect"]), _p(kp["tiles"]), _ell(kp, ellipse)))


def tile_list(kp, tx: int, ty: int, ellipse: bool = True) -> np.ndarray:
    N = kp["tiles"].shape[0]
    out = np.zeros(max(N, 1), np.uint32)
    n = lib().orc_tile_list(C.c_int(N), _p(kp["depth"]), _p(kp["rect"]), _p(kp["tiles"]), _ell(kp, ellipse),
                            C.c_int(tx), C.c_int(ty), _p(out))
    return out[:n].copy()


def lists_for_tiles(cam, kp, tiles_xy, ellipse: bool = True):
    """Brute-force per-tile lists packed as (vals, ranges) for the given tiles only
    (all other tiles empty).  Used for crops of scenes too large to bin fully."""
    ntiles = cam.tiles_x * cam.tiles_y
    ranges = np.zeros((ntiles, 2), np.uint32)
    chunks = []
    pos = 0
    for tx, ty in tiles_xy:
        ids = tile_list(kp, tx, ty, ellipse)
        t = ty * cam.tiles_x + tx
        ranges[t] = (pos, pos + len(ids))
        pos += len(ids)
        chunks.append(ids)
    vals = np.concatenate(chunks) if chunks else np.zeros(0, np.uint32)
    return vals.astype(np.uint32), ranges


def render(cam, scene, proj, vals, ranges, window=None) -> dict:
    x0, y0, x1, y1 = window if window is not None else (0, 0, cam.W, cam.H)
    ww, wh = x1 - x0, y1 - y0
    out = dict(rgb=np.zeros((3, wh, ww)), feat=np.zeros((8, wh, ww)), unc=np.zeros((wh, ww)),
               T=np.zeros((wh, ww)), n_contrib=np.zeros((wh, ww), np.int32), flip=np.zeros((wh, ww), np.uint8))
    cs = cam_struct(cam)
    vals = np.ascontiguousarray(vals, np.uint32)
    ranges = np.ascontiguousarray(ranges, np.uint32)
    feat, unc = _f32(scene.feat), _f32(scene.unc)
    lib().orc_render(C.byref(cs), C.c_int(scene.N), _p(vals), _p(ranges), _p(proj["mean2d"]), _p(proj["conic"]),
                     _p(proj["opacity"]), _p(proj["rgb"]), _p(feat), _p(unc), C.c_int(x0), C.c_int(y0),
                     C.c_int(x1), C.c_int(y1), _p(out["rgb"]), _p(out["feat"]), _p(out["unc"]), _p(out["T"]),
                     _p(out["n_contrib"]), _p(out["flip"]))
    return out


def render_bwd(cam, scene, proj, vals, ranges, dL_drgb, dL_dfeat, dL_dunc, window=None) -> dict:
    x0, y0, x1, y1 = window if window is not None else (0, 0, cam.W, cam.H)
    N = scene.N
    out = dict(mean2d=np.zeros((N, 2)), conic=np.zeros((N, 3)), opacity=np.zeros(N), rgb=np.zeros((N, 3)),
               feat=np.zeros((N, 8)), unc=np.zeros(N))
    cs = cam_struct(cam)
    vals = np.ascontiguousarray(vals, np.uint32)
    ranges = np.ascontiguousarray(ranges, np.uint32)
    feat, unc = _f32(scene.feat), _f32(scene.unc)
    g = [_f64(dL_drgb), _f64(dL_dfeat), _f64(dL_dunc)]
    lib().orc_render_bwd(C.byref(cs), C.c_int(N), _p(vals), _p(ranges), _p(proj["mean2d"]), _p(proj["conic"]),
                         _p(proj["opacity"]), _p(proj["rgb"]), _p(feat), _p(unc), C.c_int(x0), C.c_int(y0),
                         C.c_int(x1), C.c_int(y1), *[_p(a) for a in g], _p(out["mean2d"]), _p(out["conic"]),
                         _p(out["opacity"]), _p(out["rgb"]), _p(out["feat"]), _p(out["unc"]))
    return out


def decoder_fwd(feat, dec):
    """feat: [d_in, P] (any float); returns logits [N, P] in FP64."""
    feat = _f64(feat)
    d_in, P = feat.shape
    _, h1, h2, ncb = dec.dims
    logits = np.zeros((ncb, P))
    w = [_f64(a) for a in (dec.W1, dec.b1, dec.W2, dec.b2, dec.W3, dec.b3)]
    lib().orc_decoder_fwd(C.c_int(P), C.c_int(d_in), C.c_int(h1), C.c_int(h2), C.c_int(ncb), _p(feat),
                          *[_p(a) for a in w], _p(logits))
    return logits


def softmax_argmax(logits):
    logits = _f64(logits)
    ncb, P = logits.shape
    prob = np.zeros_like(logits)
    am = np.zeros(P, np.int32)
    lib().orc_softmax_argmax(C.c_int(P), C.c_int(ncb), _p(logits), _p(prob), _p(am))
    return prob, am


def decoder_loss(feat, unc, target, dec, lambda_ce=1.0, lambda_u=1.0) -> dict:
    feat = _f64(feat)
    d_in, P = feat.shape
    unc = _f64(unc).reshape(P)
    target = np.ascontiguousarray(target, np.int32).reshape(P)
    _, h1, h2, ncb = dec.dims
    out = dict(loss=np.zeros(2), d_feat=np.zeros((d_in, P)), d_unc=np.zeros(P), dW1=np.zeros((h1, d_in)),
               db1=np.zeros(h1), dW2=np.zeros((h2, h1)), db2=np.zeros(h2), dW3=np.zeros((ncb, h2)),
               db3=np.zeros(ncb))
    w = [_f64(a) for a in (dec.W1, dec.b1, dec.W2, dec.b2, dec.W3, dec.b3)]
    lib().orc_decoder_loss(C.c_int(P), C.c_int(d_in), C.c_int(h1), C.c_int(h2), C.c_int(ncb), _p(feat), _p(unc),
                           _p(target), *[_p(a) for a in w], C.c_double(lambda_ce), C.c_double(lambda_u),
                           _p(out["loss"]), _p(out["d_feat"]), _p(out["d_unc"]), _p(out["dW1"]), _p(out["db1"]),
                           _p(out["dW2"]), _p(out["db2"]), _p(out["dW3"]), _p(out["db3"]))
    return out


def query(prob, qin):
    prob = _f64(prob)
    ncb, P = prob.shape
    cb, text, negs = _f32(qin.codebook), _f32(qin.text), _f32(qin.negs)
    Q = text.shape[0]
    rel = np.zeros((Q, P))
    lib().orc_query(C.c_int(P), C.c_int(ncb), _p(prob), _p(cb), C.c_int(cb.shape[1]), C.c_int(qin.d_clip),
                    _p(text), C.c_int(Q), _p(negs), C.c_int(negs.shape[0]), _p(rel))
    return rel


def feature_map(prob, codebook):
    """F = M_infer S (supp. Sec. "Inference"): prob [N, P] -> F [P, d] in FP64."""
    prob = _f64(prob)
    ncb, P = prob.shape
    cb = _f32(codebook)
    F = np.zeros((P, cb.shape[1]))
    lib().orc_feature_map(C.c_int(P), C.c_int(ncb), _p(prob), _p(cb), C.c_int(cb.shape[1]), _p(F))
    return F


def rgb_loss(img, target, lam=0.2, want_grad=True, want_map=False) -> dict:
    """RGB loss (1 - lam) L1 + lam (1 - SSIM) on [3, H, W] images (3DGS's loss, kept by Sec. 4):
    loss = (L, L1, SSIM), grad = dL/dimg, smap = the SSIM map."""
    img, target = _f64(img), _f64(target)
    _, H, W = img.shape
    out = {"loss": np.zeros(3)}
    out["grad"] = np.zeros_like(img) if want_grad else None
    out["smap"] = np.zeros_like(img) if want_map else None
    lib().orc_rgb_loss(C.c_int(W), C.c_int(H), _p(img), _p(target), C.c_double(lam), _p(out["loss"]),
                       _p(out["grad"]) if want_grad else None, _p(out["smap"]) if want_map else None)
    return out


def l1(img, target):
    img = _f64(img)
    target = _f32(target)
    grad = np.zeros_like(img)
    loss = lib().orc_l1(C.c_int64(img.size), _p(img), _p(target), _p(grad))
    return loss, grad


def adam(param, grad, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In-place FP64 Adam step on contiguous float64 arrays."""
    for a in (param, grad, m, v):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    lib().orc_adam(C.c_int64(param.size), _p(param), _p(grad), _p(m), _p(v), C.c_int(step), C.c_double(lr),
                   C.c_double(b1), C.c_double(b2), C.c_double(eps))


# ---------------------------------------------------------------------------
def forward(scene, cam, window=None, binned=True):
    """Whole forward pass: key path, FP64 projection, binning, compositing.
    binned=False builds the per-tile lists by brute force (only the tiles the
    window touches), for scenes too large to bin in full."""
    kp = keypath(scene, cam)
    proj = project(scene, cam, kp["tiles"])
    if binned:
        keys, vals, ranges = bin(cam, kp)
    else:
        x0, y0, x1, y1 = window
        tl = [(tx, ty) for ty in range(y0 // TILE, (y1 - 1) // TILE + 1)
              for tx in range(x0 // TILE, (x1 - 1) // TILE + 1)]
        keys = None
        vals, ranges = lists_for_tiles(cam, kp, tl)
    img = render(cam, scene, proj, vals, ranges, window)
    return dict(kp=kp, proj=proj, keys=keys, vals=vals, ranges=ranges, img=img)


def bf16_bits(x) -> np.ndarray:
    """FP32 values -> BF16 bit patterns (uint16), round to nearest even."""
    x = _f32(x)
    out = np.zeros(x.shape, np.uint16)
    lib().orc_bf16_bits_array(C.c_int64(x.size), _p(x), _p(out))
    return out


def quantize(F_bf16, S, d_clip=512, lambda_d=0.5, lambda_cos=1.0, lambda_lb=0.5, round_codebook=True,
             want_D=False, want_grad=False) -> dict:
    """Quantisation of K language features against an N-entry codebook (Sec. 3.3):
    F_bf16 [K, d] uint16 BF16 bit patterns, S [N, d] codebook (FP32 values, rounded
    to BF16 when round_codebook, else used as FP64)."""
    F = np.ascontiguousarray(F_bf16, np.uint16)
    K, d = F.shape
    S64 = _f64(S)
    N = S64.shape[0]
    out = {"m": np.zeros(K, np.int32), "r": np.zeros(N), "p": np.zeros(N), "loss": np.zeros(3)}
    D = np.zeros((K, N)) if want_D else None
    G = np.zeros((N, d)) if want_grad else None
    lib().orc_quantize(C.c_int(K), C.c_int(N), C.c_int(d), C.c_int(d_clip), _p(F), _p(S64),
                       C.c_int(int(round_codebook)), C.c_double(lambda_d), C.c_double(lambda_cos),
                       C.c_double(lambda_lb), _p(D) if D is not None else None, _p(out["m"]), _p(out["r"]),
                       _p(out["p"]), _p(out["loss"]), _p(G) if G is not None else None)
    if want_D:
        out["D"] = D
    if want_grad:
        out["grad_S"] = G
    return out


SMOOTH_PARAMS = ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")


def smooth(means, feat, unc, mlp, w_s=0.1, lam=1.0) -> dict:
    """Adaptive spatial smoothing (Sec. 3.4, Eqs. eq:lem_fmlp, eq:lem_loss_mlp): s_MLP, L_smo and
    its gradients (d_feat and every MLP parameter).  mlp: object or dict with W1 [128,3], b1,
    W2 [128,128], b2, W3 [128,128], b3, W4 [8,128], b4."""
    get = (lambda k: mlp[k]) if isinstance(mlp, dict) else (lambda k: getattr(mlp, k))
    means, feat, unc = _f64(means), _f64(feat), _f64(unc)
    n = means.shape[0]
    P = [_f64(get(k)) for k in SMOOTH_PARAMS]
    out = {"s_mlp": np.zeros((n, 8)), "loss": np.zeros(1), "d_feat": np.zeros((n, 8))}
    for k, p in zip(SMOOTH_PARAMS, P):
        out["d" + k] = np.zeros_like(p)
    lib().orc_smooth(C.c_int(n), _p(means), _p(feat), _p(unc), *[_p(p) for p in P], C.c_double(w_s),
                     C.c_double(lam), _p(out["s_mlp"]), _p(out["loss"]), _p(out["d_feat"]),
                     *[_p(out["d" + k]) for k in SMOOTH_PARAMS])
    out["loss"] = float(out["loss"][0])
    return out


def densify_thresholds(grad_thresh, percent_dense, extent, min_opacity, world_frac=0.0):
    """(grad_thresh, log_big, logit_min, log_world) as FP32 values, derived in double (see
    densify.c); log_world is +inf when world-size pruning is off (world_frac <= 0)."""
    import math
    pd, ex, mo, wf = (float(np.float32(x)) for x in (percent_dense, extent, min_opacity, world_frac))
    lw = np.float32(math.log(wf * ex)) if wf > 0 else np.float32(np.inf)
    return (np.float32(grad_thresh), np.float32(math.log(pd * ex)), np.float32(math.log(mo / (1.0 - mo))), lw)


def opacity_logit(max_opacity):
    """fl(ln(m / (1 - m))) of the FP32 value m, derived in double."""
    import math
    mo = float(np.float32(max_opacity))
    return np.float32(math.log(mo / (1.0 - mo)))


def densify_stats(grad_mean2d, radius, acc, cnt, max_radius=None):
    """In place: acc [n] float32 += |dL/dmean2d|, cnt [n] int32 += 1 and max_radius [n] int32
    = max(max_radius, radius) for every Gaussian with radius > 0 (adaptive density control
    statistics).  grad_mean2d: [n, 2]."""
    g = _f32(grad_mean2d)
    r = np.ascontiguousarray(radius, np.int32)
    assert g.shape == (len(r), 2), g.shape
    assert acc.dtype == np.float32 and cnt.dtype == np.int32
    assert max_radius is None or max_radius.dtype == np.int32
    lib().orc_densify_stats(C.c_int(len(r)), _p(g), _p(r), _p(acc), _p(cnt),
                            None if max_radius is None else _p(max_radius))


def opacity_reset(opacity_raw, m, v, max_opacity=0.01):
    """In place (float32 arrays): opacity_raw = min(opacity_raw, logit(max_opacity)); m = v = 0."""
    assert opacity_raw.dtype == m.dtype == v.dtype == np.float32
    lib().orc_opacity_reset(C.c_int(len(opacity_raw)), _p(opacity_raw), _p(m), _p(v),
                            C.c_float(opacity_logit(max_opacity)))


def densify(params: dict, m: dict, v: dict, acc, cnt, noise, grad_thresh=0.0002, percent_dense=0.01, extent=1.0,
            min_opacity=0.005, max_radius=None, max_screen_size=0.0, world_frac=0.0) -> dict:
    """Adaptive density control (3DGS's, kept by Sec. 4): returns the new parameter and moment
    dicts (same field names: means, log_scales, quats, opacity_raw, sh, feat, unc) and the plan.
    max_screen_size > 0 (pixels; needs max_radius) and world_frac > 0 (fraction of extent)
    also prune Gaussians too large on screen or in the world."""
    ls = _f32(params["log_scales"])
    op = _f32(params["opacity_raw"])
    n = len(op)
    acc, cnt = _f32(acc), np.ascontiguousarray(cnt, np.int32)
    mr = None if max_radius is None else np.ascontiguousarray(max_radius, np.int32)
    assert max_screen_size <= 0 or mr is not None
    gt, lb, lm, lw = densify_thresholds(grad_thresh, percent_dense, extent, min_opacity, world_frac)
    kind = np.zeros(n, np.int32)
    total = lib().orc_densify_plan(C.c_int(n), _p(ls), _p(op), _p(acc), _p(cnt), None if mr is None else _p(mr),
                                   C.c_float(gt), C.c_float(lb), C.c_float(lm), C.c_float(max_screen_size),
                                   C.c_float(lw), _p(kind))
    keep = np.nonzero((kind == 1) | (kind == 2))[0]
    clone = np.nonzero(kind == 2)[0]
    split = np.nonzero(kind == 3)[0]
    src = np.concatenate([keep, clone, np.repeat(split, 2)])
    assert len(src) == total
    out_p, out_m, out_v = {}, {}, {}
    for k in params:
        a = np.asarray(params[k])
        out_p[k] = a[src].copy()
        z = np.zeros_like(np.asarray(m[k])[src])
        z[:len(keep)] = np.asarray(m[k])[keep]
        out_m[k] = z
        z = np.zeros_like(np.asarray(v[k])[src])
        z[:len(keep)] = np.asarray(v[k])[keep]
        out_v[k] = z
    base = len(keep) + len(clone)
    mu = np.zeros((len(split), 2, 3))
    for j, i in enumerate(split):
        for c in range(2):
            o = np.zeros(3)
            lib().orc_split_mean(_p(_f32(params["means"][i])), _p(_f32(params["log_scales"][i])),
                                 _p(_f32(params["quats"][i])), _p(_f32(noise[i, c])), _p(o))
            mu[j, c] = o
    out_p["means"] = out_p["means"].astype(np.float64)
    out_p["means"][base:] = mu.reshape(-1, 3)
    out_p["log_scales"] = out_p["log_scales"].astype(np.float64)
    out_p["log_scales"][base:] -= np.log(1.6)
    return {"params": out_p, "m": out_m, "v": out_v, "kind": kind, "n_out": int(total)}
