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
