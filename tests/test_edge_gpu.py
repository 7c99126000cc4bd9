"""Empty and degenerate inputs through the C ABI on the GPU: no Gaussians, no visible Gaussian, no pixels.

Each call must succeed, write no per-element array, and give the fixed-size outputs their value for "no
contribution": the background image with T = 1 and n_contrib = 0, zero losses and zero weight gradients.
"""
import numpy as np
import pytest
import torch

from paper_2311_18482_gb300 import synth
from parity import to_np, upstream

pytestmark = pytest.mark.gpu


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def _background_only(cam, img):
    assert np.allclose(to_np(img.rgb), np.asarray(cam.bg, np.float64)[:, None, None])
    assert np.all(to_np(img.feat) == 0) and np.all(to_np(img.unc) == 0)
    assert np.all(to_np(img.T) == 1) and np.all(to_np(img.n_contrib) == 0)


@pytest.mark.parametrize("case", ["no_gaussians", "all_culled"])
def test_lazy_binning_without_copies(leg, case):
    """le_bin_render_fwd (the training step's binning and render) with K = 0: the background, empty ranges,
    and a backward from those lists that gives zero gradients."""
    c = synth.config("c1", n=0 if case == "no_gaussians" else 64, W=48, H=40)
    sc, cam = c["scene"], c["camera"]
    cam.bg = np.array([0.25, 0.5, 0.75], np.float32)
    if case == "all_culled":
        sc.means[:, 2] = -10.0                 # behind the camera
    g = leg.Gaussians.from_scene(sc)
    proj = leg.le_preprocess(g, cam)
    ids, ranges, K, img = leg.le_bin_render_fwd(cam, proj)
    torch.cuda.synchronize()
    assert K == 0 and np.all(to_np(ranges) == 0)
    _background_only(cam, img)
    if sc.N:
        dr, df, du = upstream(np.random.default_rng(5), cam.H, cam.W)
        grads, _ = leg.le_render_bwd(cam, g, proj, ids, ranges, img, _t(dr), _t(df), _t(du))
        torch.cuda.synchronize()
        for k in ("means", "log_scales", "quats", "opacity_raw", "sh", "feat", "unc"):
            assert torch.all(getattr(grads, k) == 0), k
    leg.le_device_status()


@pytest.mark.parametrize("mode_name", ["FUSED_BF16", "UNFUSED_FP32"])
def test_decoder_without_pixels(leg, mode_name):
    """le_decode on P = 0 pixels: inference writes nothing; training sets the loss and every weight
    gradient to zero (the gradient buffers start filled with NaN here)."""
    mode = getattr(leg, mode_name)
    dec = synth.decoder_init(61, 128)
    dec_t = tuple(_t(getattr(dec, k)) for k in ("W1", "b1", "W2", "b2", "W3", "b3"))
    feat = torch.empty((8, 0), device="cuda")
    out = leg.le_decode(mode, feat, dec_t, want_prob=True)
    assert out["argmax"].numel() == 0 and out["prob"].shape == (128, 0)
    dW = [torch.full_like(t, float("nan")) for t in dec_t]
    loss = torch.full((2,), float("nan"), device="cuda")
    ws = torch.empty(max(leg.le_decode_workspace(mode | leg.DECODE_TRAIN, 0, leg.decoder_struct(*dec_t)), 1),
                     dtype=torch.uint8, device="cuda")
    leg.le_decode_raw(mode, 0, feat, torch.empty(0, device="cuda"), leg.decoder_struct(*dec_t),
                      torch.empty(0, dtype=torch.int32, device="cuda"), 1.0, 1.0, loss, torch.empty((8, 0), device="cuda"),
                      torch.empty(0, device="cuda"), leg.decoder_grads_struct(dW), None, None, None, ws)
    torch.cuda.synchronize()
    leg.le_device_status()
    assert torch.all(loss == 0)
    for g in dW:
        assert torch.all(g == 0)


def test_query_and_feature_map_without_pixels(leg):
    """le_query (fused and unfused) and le_feature_map on P = 0 pixels return without writing."""
    dec = synth.decoder_init(62, 64)
    dec_t = tuple(_t(getattr(dec, k)) for k in ("W1", "b1", "W2", "b2", "W3", "b3"))
    qin = synth.query_inputs(63, 64)
    cb, text, negs = _t(qin.codebook), _t(qin.text), _t(qin.negs)
    feat = torch.empty((8, 0), device="cuda")
    rel = leg.le_query(leg.FUSED_BF16, 0, cb, qin.d_clip, text, negs, feat=feat, dec_t=dec_t)
    assert rel.shape == (text.shape[0], 0)
    rel = leg.le_query(leg.UNFUSED_FP32, 0, cb, qin.d_clip, text, negs, dec_t=dec_t,
                       prob=torch.empty((64, 0), device="cuda"))
    assert rel.shape == (text.shape[0], 0)
    F = leg.le_feature_map(feat, dec_t, cb)
    torch.cuda.synchronize()
    leg.le_device_status()
    assert F.shape == (0, qin.codebook.shape[1])


def test_smoothing_without_gaussians(leg):
    """le_smooth on n = 0 Gaussians: zero loss and zero MLP gradients."""
    mlp = synth.smooth_mlp_init(64)
    vals = [_t(getattr(mlp, k)) for k in ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")]
    grads = [torch.full_like(v, float("nan")) for v in vals]
    e = torch.empty((0, 3), device="cuda")
    loss, d_feat, grads, _ = leg.le_smooth(e, torch.empty((0, 8), device="cuda"), torch.empty(0, device="cuda"),
                                           vals, grads=grads)
    torch.cuda.synchronize()
    leg.le_device_status()
    assert float(loss) == 0.0 and d_feat.shape == (0, 8)
    for g in grads:
        assert torch.all(g == 0)
