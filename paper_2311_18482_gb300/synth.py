"""Seeded synthetic inputs for the Language Embedded 3D Gaussians hot path.

This module only draws random numbers and lays them out; it contains none of
the method's arithmetic (no projection, no compositing, no decoding).  Both the
CUDA library's tests/bench and the FP64 oracle consume exactly these arrays.

Workloads (the paper evaluates on Mip-NeRF360 captures with CLIP/DINO targets,
Sec. 5 and supplementary Sec. "Datasets"; none of that data is available, so
seeded synthetic scenes with the paper's shapes stand in):

  c1  2,000 Gaussians, means U[-1,1]^3, 128x128, SH degree 0, seed 0
  c2  100k Gaussians from a 20-cluster mixture in [-2,2]^3, 640x480, SH deg 3,
      decoder 8->64->128->128, Voronoi index map from 30 seeds
  c3  1M Gaussians, 50 clusters, 1296x840, SH deg 3, uncertainty U[0,1]
  c4  3M Gaussians, 50 clusters, 1920x1080, codebook 256 x 896 (512+384),
      4 text embeddings and 4 canonical negatives (random unit 512-vectors)
  c5  1M Gaussians, 16 poses on a circle of radius 3, 1296x840, per-view
      Voronoi maps (128-entry codebook), uncertainty initialised to 0
  quantisation (Sec. 3.3): per-pixel hybrid features F = [CLIP 512 | DINO 384]
      of one 1296x840 view drawn around the codes of a hidden 128-entry set
      (one per Voronoi region of the view, Gaussian noise per pixel), stored as
      BF16; the codebook being optimised starts from 128 random features

Per-Gaussian parameters are FP32 structure-of-arrays:
  means [N,3], log_scales [N,3], quats [N,4] (w,x,y,z), opacity_raw [N]
  (opacity = sigmoid(opacity_raw)), sh [N,(deg+1)^2,3], feat [N,8], unc [N].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

D_FEAT = 8          # compact semantic feature width d_s (Sec. 4)
TILE = 16           # screen tile edge in pixels


@dataclass
class Camera:
    """Pinhole camera, OpenCV axes (x right, y down, z forward).

    view is the 3x4 world-to-camera matrix [R | t], row-major.  Pixel (i, j)
    is sampled at integer coordinates; cx = (W-1)/2, cy = (H-1)/2.
    """
    view: np.ndarray            # float32 [12]
    campos: np.ndarray          # float32 [3]
    fx: float
    fy: float
    cx: float
    cy: float
    W: int
    H: int
    near: float = 0.2
    bg: np.ndarray = field(default_factory=lambda: np.zeros(3, np.float32))

    @property
    def tiles_x(self) -> int:
        return (self.W + TILE - 1) // TILE

    @property
    def tiles_y(self) -> int:
        return (self.H + TILE - 1) // TILE


def look_at_camera(eye, target, up, W, H, fov_x_deg, near=0.2, bg=(0.0, 0.0, 0.0)) -> Camera:
    """World-to-camera matrix for a camera at `eye` looking at `target`."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    x = np.cross(f, np.asarray(up, np.float64))
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    R = np.stack([x, y, f])                 # rows: camera axes in world coords
    t = -R @ eye
    view = np.concatenate([R, t[:, None]], axis=1).astype(np.float32).reshape(12)
    fx = (W / 2.0) / math.tan(math.radians(fov_x_deg) / 2.0)
    return Camera(view=view, campos=eye.astype(np.float32), fx=float(np.float32(fx)),
                  fy=float(np.float32(fx)), cx=(W - 1) / 2.0, cy=(H - 1) / 2.0, W=W, H=H,
                  near=near, bg=np.asarray(bg, np.float32))


def circle_pose(k: int, n_poses: int, W: int, H: int, radius: float = 3.0, fov_x_deg: float = 60.0) -> Camera:
    """Pose k of n on the circle of given radius in the y=0 plane, looking at the origin."""
    a = 2.0 * math.pi * k / n_poses
    eye = (radius * math.cos(a), 0.0, radius * math.sin(a))
    return look_at_camera(eye, (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), W, H, fov_x_deg)


@dataclass
class Scene:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_raw: np.ndarray
    sh: np.ndarray              # [N, (deg+1)^2, 3]
    feat: np.ndarray            # [N, 8]
    unc: np.ndarray             # [N]
    sh_degree: int

    @property
    def N(self) -> int:
        return self.means.shape[0]


def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def uniform_cube_scene(seed: int = 0, n: int = 2000) -> Scene:
    """Config c1: means U[-1,1]^3, log-scales N(-3,0.5), random unit quaternions,
    opacity_raw N(0,1), SH degree 0 whose DC coefficient is U[-sqrt(pi), sqrt(pi)]
    (so that the degree-0 colour is uniform in [0,1]), feat N(0,1)^8, unc U[0,1]."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1.0, 1.0, (n, 3)).astype(np.float32)
    log_scales = rng.normal(-3.0, 0.5, (n, 3)).astype(np.float32)
    quats = _unit_quats(rng, n)
    opacity_raw = rng.standard_normal(n).astype(np.float32)
    sp = math.sqrt(math.pi)
    sh = rng.uniform(-sp, sp, (n, 1, 3)).astype(np.float32)
    feat = rng.standard_normal((n, D_FEAT)).astype(np.float32)
    unc = rng.uniform(0.0, 1.0, n).astype(np.float32)
    return Scene(means, log_scales, quats, opacity_raw, sh, feat, unc, 0)


def cluster_scene(seed: int, n: int, n_clusters: int, sh_degree: int = 3, unc: str = "uniform") -> Scene:
    """Configs c2-c5: Gaussian mixture with centres U[-2,2]^3, isotropic sigma 0.25,
    equal weights, clipped to [-2,2]^3; SH coefficients N(0,0.1)."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-2.0, 2.0, (n_clusters, 3))
    which = rng.integers(0, n_clusters, n)
    means = np.clip(centres[which] + rng.normal(0.0, 0.25, (n, 3)), -2.0, 2.0).astype(np.float32)
    log_scales = rng.normal(-3.0, 0.5, (n, 3)).astype(np.float32)
    quats = _unit_quats(rng, n)
    opacity_raw = rng.standard_normal(n).astype(np.float32)
    nc = (sh_degree + 1) ** 2
    sh = rng.normal(0.0, 0.1, (n, nc, 3)).astype(np.float32)
    feat = rng.standard_normal((n, D_FEAT)).astype(np.float32)
    if unc == "uniform":
        u = rng.uniform(0.0, 1.0, n).astype(np.float32)
    else:
        u = np.zeros(n, np.float32)
    return Scene(means, log_scales, quats, opacity_raw, sh, feat, u, sh_degree)


@dataclass
class Decoder:
    """Per-pixel MLP weights, [out, in] row-major (a 1x1 convolution), FP32."""
    W1: np.ndarray
    b1: np.ndarray
    W2: np.ndarray
    b2: np.ndarray
    W3: np.ndarray
    b3: np.ndarray

    @property
    def dims(self):
        return (self.W1.shape[1], self.W1.shape[0], self.W2.shape[0], self.W3.shape[0])


def decoder_init(seed: int, n_cb: int, h1: int = 64, h2: int = 128, d_in: int = D_FEAT) -> Decoder:
    """Kaiming-uniform style init: weights and biases U[-1/sqrt(fan_in), 1/sqrt(fan_in)]."""
    rng = np.random.default_rng(seed)
    out = []
    for fi, fo in ((d_in, h1), (h1, h2), (h2, n_cb)):
        bound = 1.0 / math.sqrt(fi)
        out.append(rng.uniform(-bound, bound, (fo, fi)).astype(np.float32))
        out.append(rng.uniform(-bound, bound, fo).astype(np.float32))
    return Decoder(*out)


def voronoi_index_map(seed: int, W: int, H: int, n_cb: int, n_seeds: int = 30) -> np.ndarray:
    """Synthetic semantic index map: each pixel takes the codebook id of the nearest of
    n_seeds random seed points (Euclidean pixel distance, ties to the lowest seed)."""
    rng = np.random.default_rng(seed)
    sx = rng.uniform(0.0, W, n_seeds)
    sy = rng.uniform(0.0, H, n_seeds)
    ids = rng.integers(0, n_cb, n_seeds).astype(np.int32)
    out = np.empty((H, W), np.int32)
    xs = np.arange(W, dtype=np.float64)
    for y0 in range(0, H, 64):
        ys = np.arange(y0, min(H, y0 + 64), dtype=np.float64)
        d2 = (xs[None, None, :] - sx[:, None, None]) ** 2 + (ys[None, :, None] - sy[:, None, None]) ** 2
        out[y0:y0 + len(ys)] = ids[np.argmin(d2, axis=0)]
    return out


def smooth_rgb_target(seed: int, W: int, H: int) -> np.ndarray:
    """A smooth random RGB target image [3,H,W] in [0,1] (sum of random sinusoids)."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    img = np.zeros((3, H, W))
    for c in range(3):
        for _ in range(4):
            kx, ky = rng.uniform(-6, 6, 2) * 2 * math.pi
            ph = rng.uniform(0, 2 * math.pi)
            img[c] += np.sin(kx * xx / W + ky * yy / H + ph)
    img = 0.5 + 0.125 * img
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def unit_rows(rng, n, d) -> np.ndarray:
    v = rng.standard_normal((n, d))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v.astype(np.float32)


@dataclass
class QueryInputs:
    codebook: np.ndarray        # [n_cb, d] unit rows (d = 512 + 384)
    text: np.ndarray            # [Q, d_clip] unit rows
    negs: np.ndarray            # [n_neg, d_clip] unit rows
    d_clip: int


def query_inputs(seed: int, n_cb: int = 256, d_clip: int = 512, d_dino: int = 384,
                 n_text: int = 4, n_neg: int = 4) -> QueryInputs:
    rng = np.random.default_rng(seed)
    cb = unit_rows(rng, n_cb, d_clip + d_dino)
    text = unit_rows(rng, n_text, d_clip)
    negs = unit_rows(rng, n_neg, d_clip)
    return QueryInputs(cb, text, negs, d_clip)


# ---------------------------------------------------------------------------
# The five workloads.  `n`, `W`, `H` overrides give smaller cases with the same
# distributions (used by the parity tests).

def config(name: str, n: int | None = None, W: int | None = None, H: int | None = None, pose: int = 0):
    """Returns dict(scene, camera, [decoder, target_idx, rgb_target, query]) for a workload."""
    if name == "c1":
        W = W or 128
        H = H or 128
        scene = uniform_cube_scene(0, 2000 if n is None else n)
        cam = look_at_camera((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), W, H, 60.0)
        return dict(scene=scene, camera=cam)
    if name == "c2":
        W = W or 640
        H = H or 480
        scene = cluster_scene(1, 100_000 if n is None else n, 20)
        cam = circle_pose(pose, 16, W, H)
        dec = decoder_init(101, 128)
        return dict(scene=scene, camera=cam, decoder=dec, target_idx=voronoi_index_map(1001 + pose, W, H, 128),
                    rgb_target=smooth_rgb_target(2001 + pose, W, H))
    if name == "c3":
        W = W or 1296
        H = H or 840
        scene = cluster_scene(2, 1_000_000 if n is None else n, 50)
        cam = circle_pose(pose, 16, W, H)
        return dict(scene=scene, camera=cam)
    if name == "c4":
        W = W or 1920
        H = H or 1080
        scene = cluster_scene(3, 3_000_000 if n is None else n, 50)
        cam = circle_pose(pose, 16, W, H)
        dec = decoder_init(103, 256)
        return dict(scene=scene, camera=cam, decoder=dec, query=query_inputs(303, 256))
    if name == "c5":
        W = W or 1296
        H = H or 840
        scene = cluster_scene(4, 1_000_000 if n is None else n, 50, unc="zero")
        cam = circle_pose(pose, 16, W, H)
        dec = decoder_init(104, 128)
        return dict(scene=scene, camera=cam, decoder=dec,
                    target_idx=voronoi_index_map(1000 + pose, W, H, 128),
                    rgb_target=smooth_rgb_target(2000 + pose, W, H))
    raise ValueError(f"unknown workload {name!r}")


def _bf16_bits(x: np.ndarray) -> np.ndarray:
    """FP32 -> BF16 bit patterns (round to nearest even), for storing synthetic features."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32)
    return ((u + np.uint32(0x7FFF) + ((u >> np.uint32(16)) & np.uint32(1))) >> np.uint32(16)).astype(np.uint16)


def quant_inputs(seed: int, K: int, n_cb: int = 128, d_clip: int = 512, d_dino: int = 384, n_hidden: int = 128,
                 noise: float = 0.6, W: int | None = None):
    """Synthetic language features for the quantisation stage: K features
    [K, d_clip + d_dino] as BF16 bit patterns around n_hidden hidden unit codes
    (per part), each feature's code chosen by a Voronoi map of the pixel grid of
    width W (or uniformly at random when W is None), plus N(0, noise^2/d) per
    dimension; and an n_cb x d FP32 codebook initialised from random features."""
    rng = np.random.default_rng(seed)
    d = d_clip + d_dino
    centres = np.concatenate([unit_rows(rng, n_hidden, d_clip), unit_rows(rng, n_hidden, d_dino)], axis=1)
    if W is None:
        lab = rng.integers(0, n_hidden, K)
    else:
        H = (K + W - 1) // W
        lab = voronoi_index_map(seed + 1, W, H, n_hidden, n_seeds=60).reshape(-1)[:K]
    F = centres[lab] + rng.standard_normal((K, d)).astype(np.float32) * np.float32(noise / math.sqrt(d))
    S = F[rng.choice(K, n_cb, replace=K < n_cb)].astype(np.float32)
    return _bf16_bits(F), S


@dataclass
class SmoothMLP:
    """MLP of the adaptive spatial smoothing (supp. Tab. pemlp): 3 -> 128 -> 128 -> 128 -> 8,
    FP32 weights [out][in]."""
    W1: np.ndarray
    b1: np.ndarray
    W2: np.ndarray
    b2: np.ndarray
    W3: np.ndarray
    b3: np.ndarray
    W4: np.ndarray
    b4: np.ndarray


def smooth_mlp_init(seed: int) -> SmoothMLP:
    """Kaiming-uniform weights and small uniform biases (PyTorch's Linear default scheme)."""
    rng = np.random.default_rng(seed)
    dims = [(3, 128), (128, 128), (128, 128), (128, 8)]
    ws = []
    for fi, fo in dims:
        bound = 1.0 / math.sqrt(fi)
        ws.append(rng.uniform(-bound, bound, (fo, fi)).astype(np.float32))
        ws.append(rng.uniform(-bound, bound, fo).astype(np.float32))
    return SmoothMLP(*ws)
