"""One training step of the Language Embedded 3D Gaussians hot path on one GPU,
driven entirely through the C ABI with preallocated device buffers:

  le_preprocess -> le_bin_render_fwd (binning + compositing, lazily placed)
  -> le_decode_l1 (D_MLP + uncertainty-weighted CE + L_u, Eqs. 8-12, training
     mode, with the RGB L1 term of Sec. 4 in the same pass; or le_rgb_loss with
     D-SSIM and le_decode)
  -> le_render_bwd_screen (screen-space gradients) -> le_project_bwd_adam
     (all Gaussian parameter gradients, each applied by Adam where it is
     computed; u clamped to [0,1], Sec. 3.4.2)
  -> le_adam (decoder parameters)

With fused_adam=False the Gaussian gradients are written out by le_render_bwd
and le_adam runs over them (bit-identical result, more memory traffic).
All parameters live in one flat FP32 buffer (each tensor a 16-byte aligned
view), so Adam is two launches over contiguous memory.  The loss weights are
the paper's (all lambda = 1, Sec. 4).
"""
from __future__ import annotations

import torch

from . import binding as B

_FIELDS = ("means", "log_scales", "quats", "opacity_raw", "sh", "feat")
_DEC = ("W1", "b1", "W2", "b2", "W3", "b3")


def _pad4(n):
    return (n + 3) // 4 * 4


class FlatParams:
    """Views of the Gaussian and decoder parameters in one flat buffer; unc last."""

    def __init__(self, scene, dec, device):
        N = scene.N
        shapes = {"means": (N, 3), "log_scales": (N, 3), "quats": (N, 4), "opacity_raw": (N,),
                  "sh": (N, scene.sh.shape[1], 3), "feat": (N, 8)}
        for k in _DEC:
            shapes[k] = getattr(dec, k).shape
        shapes["unc"] = (N,)
        self.order = list(_FIELDS) + list(_DEC) + ["unc"]
        self.offsets, off = {}, 0
        for k in self.order:
            n = 1
            for d in shapes[k]:
                n *= d
            self.offsets[k] = (off, n, shapes[k])
            off = _pad4(off + n)
        self.total = off
        self.unc_offset = self.offsets["unc"][0]
        self.sh_degree = scene.sh_degree
        self.device = device

    def views(self, flat):
        return {k: flat[o:o + n].view(*shp) for k, (o, n, shp) in self.offsets.items()}


class TrainState:
    def __init__(self, scene, dec, W, H, device="cuda", decoder_mode=B.FUSED_BF16, lr=1e-3, fused_adam=True,
                 rgb_loss="l1", lambda_ssim=0.2):
        self.layout = FlatParams(scene, dec, device)
        L = self.layout
        self.params = torch.zeros(L.total, dtype=torch.float32, device=device)
        self.grads = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        pv = L.views(self.params)
        src = {k: getattr(scene, k) for k in list(_FIELDS) + ["unc"]}
        src.update({k: getattr(dec, k) for k in _DEC})
        for k, t in pv.items():
            t.copy_(torch.from_numpy(src[k]).reshape(t.shape))
        self.pv, self.gv = pv, L.views(self.grads)
        self.g = B.Gaussians(pv["means"], pv["log_scales"], pv["quats"], pv["opacity_raw"], pv["sh"], pv["feat"],
                             pv["unc"], scene.sh_degree)
        self.gg = B.grads_struct(B.Gaussians(*(self.gv[k] for k in list(_FIELDS) + ["unc"]), scene.sh_degree))
        self.dec = B.decoder_struct(*(pv[k] for k in _DEC))
        self.dgrad = B.decoder_grads_struct([self.gv[k] for k in _DEC])
        mv, vv = L.views(self.m), L.views(self.v)
        gfields = list(_FIELDS) + ["unc"]
        self.gm = B.Gaussians(*(mv[k] for k in gfields), scene.sh_degree)
        self.gvv = B.Gaussians(*(vv[k] for k in gfields), scene.sh_degree)
        self.fused_adam = fused_adam
        self.dec_lo = L.offsets["W1"][0]
        N, P = scene.N, W * H
        self.W, self.H, self.P = W, H, P
        self.proj = B.Projected.empty(N, device)
        self.bins = B.BinSortBuffers()
        self.img = B.Image.empty(H, W, device)
        self.loss = torch.zeros(3, dtype=torch.float32, device=device)     # L1, L_CE, L_u
        self.d_rgb = torch.empty((3, H, W), dtype=torch.float32, device=device)
        self.d_feat = torch.empty((8, H, W), dtype=torch.float32, device=device)
        self.d_unc = torch.empty((H, W), dtype=torch.float32, device=device)
        self.grad2d = torch.empty((N, B.SPLAT_STRIDE), dtype=torch.float32, device=device)
        self.mode = decoder_mode
        self.dec_ws = torch.empty(max(B.le_decode_workspace(decoder_mode | B.DECODE_TRAIN, P, self.dec), 1),
                                  dtype=torch.uint8, device=device)
        self.step_count = 0
        self.lr = lr
        # RGB loss: "l1" (the training-loop configuration) or "l1_dssim", 3DGS's (1 - lambda) L1 +
        # lambda D-SSIM that Sec. 4 keeps; loss[0] then holds the combined value
        self.rgb_loss, self.lambda_ssim = rgb_loss, lambda_ssim
        self.rgb_ws = torch.empty(B.le_rgb_loss_workspace(W, H), dtype=torch.uint8, device=device) \
            if rgb_loss == "l1_dssim" else None
        self.rgb_terms = torch.empty(3, dtype=torch.float32, device=device)
        self.K = 0
        self.events = None

    def state_dict(self):
        """Everything a resumed run needs: parameters, Adam moments, step count."""
        return {"params": self.params.detach().cpu().clone(), "m": self.m.detach().cpu().clone(),
                "v": self.v.detach().cpu().clone(), "step": self.step_count}

    def load_state_dict(self, sd):
        self.params.copy_(sd["params"])
        self.m.copy_(sd["m"])
        self.v.copy_(sd["v"])
        self.step_count = int(sd["step"])

    def _mark(self, name):
        if self.events is not None:
            ev = torch.cuda.Event(enable_timing=True)
            ev.record()
            self.events.append((name, ev))

    def step(self, cam, rgb_target, idx_target):
        """One fwd+bwd+Adam step on view `cam`; returns the device loss vector (L1, L_CE, L_u)."""
        self._mark("start")
        B.le_preprocess(self.g, cam, self.proj)
        self._mark("preprocess")
        ids, ranges, self.K, _ = B.le_bin_render_fwd(cam, self.proj, self.bins, self.img)
        self._mark("bin_render")
        if self.rgb_loss == "l1_dssim":
            B.le_rgb_loss(self.img.rgb, rgb_target, self.lambda_ssim, loss=self.rgb_terms, grad=self.d_rgb,
                          workspace=self.rgb_ws)
            self.loss[0:1].copy_(self.rgb_terms[0:1])
            B.le_decode_raw(self.mode, self.P, self.img.feat, self.img.unc, self.dec, idx_target, 1.0, 1.0,
                            self.loss[1:3], self.d_feat, self.d_unc, self.dgrad, None, None, None, self.dec_ws)
        else:
            # the L1 term rides in the decoder's training pass (one launch fewer with the fused decoder)
            B.le_decode_l1_raw(self.mode, self.P, self.img.feat, self.img.unc, self.dec, idx_target, 1.0, 1.0,
                               self.loss[1:3], self.d_feat, self.d_unc, self.dgrad, self.img.rgb, rgb_target,
                               self.loss[0:1], self.d_rgb, self.dec_ws)
        self._mark("decoder")
        self.step_count += 1
        u0, d0 = self.layout.unc_offset, self.dec_lo
        if self.fused_adam:
            # le_render_bwd_adam in its two halves (identical results), so the
            # stages can be timed apart
            B.le_render_bwd_screen(cam, self.g, self.proj, ids, ranges, self.img, self.d_rgb, self.d_feat,
                                   self.d_unc, grad2d=self.grad2d)
            self._mark("render_bwd")
            # the decoder parameters' Adam step rides in the same launch (their gradients are complete:
            # le_decode wrote them before the render backward)
            B.le_project_bwd_adam_extra(cam, self.g, self.proj, self.grad2d, self.gm, self.gvv, self.step_count,
                                        self.params[d0:u0], self.grads[d0:u0], self.m[d0:u0], self.v[d0:u0],
                                        lr=self.lr)
            self._mark("project_bwd_adam")
        else:
            cs, gs, ps = B.camera_struct(cam), self.g.struct(), self.proj.struct()
            import ctypes as C
            B._check(B.load().le_render_bwd(C.byref(cs), C.byref(gs), C.byref(ps), B._ptr(ids), B._ptr(ranges),
                                            B._ptr(self.img.T), B._ptr(self.img.n_contrib), B._ptr(self.d_rgb),
                                            B._ptr(self.d_feat), B._ptr(self.d_unc), B._ptr(self.grad2d),
                                            C.byref(self.gg), B._stream()))
            self._mark("render_bwd")
            B.le_adam(self.params[:u0], self.grads[:u0], self.m[:u0], self.v[:u0], self.step_count, lr=self.lr)
            B.le_adam(self.params[u0:], self.grads[u0:], self.m[u0:], self.v[u0:], self.step_count, lr=self.lr,
                      clamp_lo=0.0, clamp_hi=1.0)
        self._mark("adam")
        return self.loss
