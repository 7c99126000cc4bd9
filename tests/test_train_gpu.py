"""The fused training step: le_render_bwd_adam applies Adam where each Gaussian
gradient is computed, and must agree with le_render_bwd followed by le_adam.

The Adam update is one fixed operation sequence on both paths; the gradient
code is compiled once per path, and the compiler may contract a multiply-add
differently in each copy, so a gradient can differ in its last bits.
  1. Gradients: one step with lr = 0 leaves the parameters unchanged and the
     first moment is (1 - beta1) g on both paths; per field, |dm| must stay
     within 1e-4 of the field's largest |m| -- the bar of the rasterizer's
     gradient parity (the screen-space gradients are summed with atomic adds
     whose order varies from run to run, and the quaternion gradient's
     tangent projection cancels, so runs differ by up to ~1e-5 of the field's
     scale; a wrong element or field would differ by O(1)) -- and the
     parameters must be identical.
  2. Training: three steps on both paths; the losses of every step agree to
     1e-4 relative (small differences change later renders a little), u stays
     in [0, 1].
"""
import numpy as np
import pytest
import torch

from paper_2311_18482_gb300 import synth

pytestmark = pytest.mark.gpu


def _state(fused, lr=1e-3):
    from paper_2311_18482_gb300.training import TrainState
    c = synth.config("c2", n=20000, W=320, H=240)
    return TrainState(c["scene"], c["decoder"], 320, 240, fused_adam=fused, lr=lr)


def _targets():
    rgb = torch.from_numpy(synth.smooth_rgb_target(7, 320, 240)).cuda()
    idx = torch.from_numpy(synth.voronoi_index_map(8, 320, 240, 128)).cuda()
    return rgb, idx


def test_fused_adam_gradients_match(leg):
    a, b = _state(False, lr=0.0), _state(True, lr=0.0)
    rgb, idx = _targets()
    cam = synth.circle_pose(1, 4, 320, 240)
    for st in (a, b):
        st.step(cam, rgb, idx)
    torch.cuda.synchronize()
    assert torch.equal(a.params, b.params)
    va, vb = a.layout.views(a.m), b.layout.views(b.m)
    for k in va:
        d = (va[k] - vb[k]).abs()
        scale = va[k].abs().max().clamp_min(1e-30)
        print(f"m.{k}: max |diff| / max |m| {float(d.max() / scale):.2e}, identical {float((d == 0).float().mean()):.4f}")
        assert float(d.max()) <= 1e-4 * float(scale), k
    assert float(va["means"].abs().max()) > 0


def test_fused_adam_training_matches(leg):
    a, b = _state(False), _state(True)
    rgb, idx = _targets()
    for k in range(3):
        cam = synth.circle_pose(k, 4, 320, 240)
        la, lb = a.step(cam, rgb, idx).clone(), b.step(cam, rgb, idx).clone()
        torch.cuda.synchronize()
        assert torch.allclose(la, lb, rtol=1e-4, atol=1e-7), (k, la, lb)
    u = b.layout.views(b.params)["unc"]
    assert float(u.min()) >= 0.0 and float(u.max()) <= 1.0
    c = synth.config("c2", n=20000, W=320, H=240)
    assert not np.array_equal(b.layout.views(b.params)["means"].cpu().numpy(), c["scene"].means)


def test_fused_adam_rejects_bad_config(leg):
    import paper_2311_18482_gb300.binding as B
    st = _state(True)
    cam = synth.circle_pose(0, 4, 320, 240)
    with pytest.raises(B.LegError) as e:
        B.le_render_bwd_adam(cam, st.g, st.proj, torch.zeros(1, dtype=torch.int32, device="cuda"),
                             torch.zeros((cam.tiles_x * cam.tiles_y, 2), dtype=torch.int32, device="cuda"), st.img,
                             st.d_rgb, st.d_feat, st.d_unc, st.gm, st.gvv, step=0)
    assert e.value.status == B.LE_ERR_INVALID_ARG


_F = ("means", "log_scales", "quats", "opacity_raw", "sh", "feat", "unc")


@pytest.mark.parametrize("n", [20003, 4096])
def test_backward_halves_match_single_calls(leg, n):
    """le_render_bwd_screen + le_project_bwd(_adam) against le_render_bwd and
    le_project_bwd + le_adam, with a partly filled last warp (n = 20003) and
    full warps only (n = 4096).  Given the same grad2d, the projection half's
    gradients equal le_render_bwd's (the same kernel); its fused Adam step
    equals le_adam over those gradients within a last-bit contraction
    difference of the gradient (1e-5 of each field's scale)."""
    import paper_2311_18482_gb300.binding as B
    from parity import upstream
    c = synth.config("c2", n=n, W=320, H=240)
    sc, cam = c["scene"], c["camera"]
    g = B.Gaussians.from_scene(sc)
    proj = B.le_preprocess(g, cam)
    ids, ranges, K, img = B.le_bin_render_fwd(cam, proj)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    dr, df, du = (t(a) for a in upstream(np.random.default_rng(21), cam.H, cam.W))
    grads_a, g2a = B.le_render_bwd(cam, g, proj, ids, ranges, img, dr, df, du)
    g2b = B.le_render_bwd_screen(cam, g, proj, ids, ranges, img, dr, df, du)
    torch.cuda.synchronize()
    # screen-space gradients: same kernel, atomic summation order may differ
    assert float((g2a - g2b).abs().max()) <= 1e-5 * float(g2a.abs().max())
    grads_b = B.le_project_bwd(cam, g, proj, g2a)
    for k in _F:
        assert torch.equal(getattr(grads_a, k), getattr(grads_b, k)), k
    # fused Adam from the same grad2d vs le_adam over the written gradients
    rng = np.random.default_rng(22)
    m0 = {k: t(rng.standard_normal(getattr(g, k).shape) * 1e-3) for k in _F}
    v0 = {k: t(rng.uniform(0, 1e-5, getattr(g, k).shape)) for k in _F}
    ga = B.Gaussians(*(getattr(g, k).clone() for k in _F), g.sh_degree)
    gb = B.Gaussians(*(getattr(g, k).clone() for k in _F), g.sh_degree)
    ma = B.Gaussians(*(m0[k].clone() for k in _F), g.sh_degree)
    va = B.Gaussians(*(v0[k].clone() for k in _F), g.sh_degree)
    mb = B.Gaussians(*(m0[k].clone() for k in _F), g.sh_degree)
    vb = B.Gaussians(*(v0[k].clone() for k in _F), g.sh_degree)
    B.le_project_bwd_adam(cam, ga, proj, g2a, ma, va, step=3)
    for k in _F:
        lo, hi = (0.0, 1.0) if k == "unc" else (-float("inf"), float("inf"))
        B.le_adam(getattr(gb, k).view(-1), getattr(grads_a, k).view(-1), getattr(mb, k).view(-1),
                  getattr(vb, k).view(-1), 3, clamp_lo=lo, clamp_hi=hi)
    torch.cuda.synchronize()
    for k in _F:
        for x, y in ((ga, gb), (ma, mb), (va, vb)):
            a, b = getattr(x, k), getattr(y, k)
            assert float((a - b).abs().max()) <= 1e-5 * max(float(b.abs().max()), 1e-6), k
    assert float(ga.unc.min()) >= 0.0 and float(ga.unc.max()) <= 1.0
    assert not torch.equal(ga.means, g.means)
    # the same projection Adam with one more flat range in the launch (25,001 elements: quads and a tail):
    # the Gaussians as without it, the range bit for bit as le_adam leaves it
    n_x = 25001
    px, gx = t(rng.standard_normal(n_x)), t(rng.standard_normal(n_x) * 1e-2)
    mx, vx = t(rng.standard_normal(n_x) * 1e-3), t(rng.uniform(0, 1e-5, n_x))
    gc = B.Gaussians(*(getattr(g, k).clone() for k in _F), g.sh_degree)
    mc = B.Gaussians(*(m0[k].clone() for k in _F), g.sh_degree)
    vc = B.Gaussians(*(v0[k].clone() for k in _F), g.sh_degree)
    pxa, mxa, vxa = px.clone(), mx.clone(), vx.clone()
    B.le_project_bwd_adam_extra(cam, gc, proj, g2a, mc, vc, 3, pxa, gx, mxa, vxa)
    B.le_adam(px, gx, mx, vx, 3)
    torch.cuda.synchronize()
    for k in _F:
        for x, y in ((ga, gc), (ma, mc), (va, vc)):
            assert torch.equal(getattr(x, k), getattr(y, k)), k
    assert torch.equal(pxa, px) and torch.equal(mxa, mx) and torch.equal(vxa, vx)


def test_training_step_ragged_view(leg):
    """The whole training step on a view whose size is no multiple of anything the kernels tile by:
    333 x 217 pixels (partial 16 x 16 tiles on both edges; 72,261 pixels, so the decoder's last
    128-pixel tile holds 69), 6,000 Gaussians of SH degree 1.  The fused BF16 and the unfused FP32
    decoder paths render identically, agree on the first step's losses (L1 to the order of its block
    sums, CE and L_u within the fused decoder's BF16 bounds) and stay within 1e-3 over two more steps; u stays in [0, 1]."""
    from paper_2311_18482_gb300.training import TrainState
    W, H = 333, 217
    sc = synth.cluster_scene(11, 6000, 12, sh_degree=1)
    dec = synth.decoder_init(12, 128)
    rgb = torch.from_numpy(synth.smooth_rgb_target(13, W, H)).cuda()
    idx = torch.from_numpy(synth.voronoi_index_map(14, W, H, 128)).cuda()
    a = TrainState(sc, dec, W, H, decoder_mode=leg.FUSED_BF16)
    b = TrainState(sc, dec, W, H, decoder_mode=leg.UNFUSED_FP32)
    for k in range(3):
        cam = synth.circle_pose(k, 4, W, H)
        la, lb = a.step(cam, rgb, idx).clone(), b.step(cam, rgb, idx).clone()
        torch.cuda.synchronize()
        if k == 0:
            assert torch.equal(a.img.rgb, b.img.rgb) and torch.equal(a.img.feat, b.img.feat)
            # equal images; the L1 loss is the sum of one FP32 partial per block of le_rgb_l1 (at most 152 x 8
            # blocks of 256 elements) added atomically in any order: two orders of m nonnegative terms differ
            # by at most 2 (m - 1) u of their sum (u = 2^-24)
            m_blocks = min((3 * W * H + 255) // 256, 152 * 8)
            assert abs(float(la[0]) - float(lb[0])) <= 2 * (m_blocks - 1) * 2.0 ** -24 * abs(float(lb[0]))
            assert torch.allclose(la[1:], lb[1:], rtol=2e-4, atol=1e-7), (la, lb)
        else:
            assert torch.allclose(la, lb, rtol=1e-3, atol=1e-6), (k, la, lb)
    leg.le_device_status()
    for st in (a, b):
        u = st.layout.views(st.params)["unc"]
        assert float(u.min()) >= 0.0 and float(u.max()) <= 1.0
