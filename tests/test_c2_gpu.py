"""The decoder-training workload at its stated size (100k Gaussians from a 20-cluster
mixture, SH degree 3, 640x480, decoder 8->64->128 -> 128 codes, Voronoi index map
from 30 seeds), and the differentiation workload's finite-difference check on the
GPU at 1M Gaussians.

1. One full training step -- preprocess, binning + compositing, RGB L1, decoder loss
   (Eqs. eq:lem_loss_ce1, eq:lem_loss_uncer), compositing and projection adjoints --
   with the unfused FP32 decoder, against the FP64 oracle on the 64x64 centre crop:
   the GPU's upstream gradients are kept on the crop only, so both sides
   differentiate the same loss.  Bars: images 1e-4, upstream gradients and all
   parameter gradients 1e-4 (per-tensor infinity norm relative to the tensor's
   scale), flip pixels (on an alpha threshold) and pixels whose L1 sign is within
   1e-5 of zero left out on both sides.
2. The fused BF16 decoder against the unfused FP32 one on the whole view, with the
   bars derived for the BF16 operands (relative Frobenius: loss 1e-4, d_unc 1e-3,
   layer 3 2e-2, layer 2 8e-2, layer 1 and d_feat 1e-1), and the Gaussian gradients
   they drive (1e-1: every channel of the upstream gradient but RGB passes through
   d_feat or d_unc).
3. Training with the repo's kernels (1000 fused steps, Adam lr 1e-3), then on the
   rendered 640x480 view: the fused BF16 argmax agrees with the FP64 argmax of the
   same features on >= 99.9 % of pixels, and every disagreement is a near tie (the
   FP64 logit of the GPU's choice within 0.5 of the maximum: BF16 rounds each MMA
   operand to 2^-9 relative, and the trained logits reach |z| ~ 30); the trained
   decoder's accuracy against the index map beats a non-learned decoding of the same
   rendered features -- the nearest per-class mean feature, fitted on the same
   pixels -- by >= 3 points, with at most a fifth of its errors.
4. Central differences on the GPU at 1M Gaussians (1296x840): 64 randomly chosen
   Gaussians that reach at least one pixel (3,693 of the 1M do on this view), one
   random direction in each parameter group (mean in the image plane, log-scales,
   quaternion, opacity, SH, feature, uncertainty).  The loss is a smooth random
   linear functional of the rendered channels, times, per Gaussian i, a fixed
   mask that is 0 where i's alpha (at the unperturbed parameters) is below 2/255
   and 1 above 4/255.  Without the mask a geometric perturbation moves i's
   alpha = 1/255 contour, every pixel it crosses adds a jump of about T c / 255
   that the derivative of the smooth pieces leaves out, and those jumps grow with
   h as the signal does (1-10 % of the difference, measured); with the mask the
   crossed pixels carry no weight, and the analytic gradient is taken for the
   same masked functional.  Bars: relative L2 error over the 64 samples <= 2e-2
   (geometric groups; the remaining jumps are transmittance-cutoff crossings of
   about 1e-4 c each) and <= 1e-3 (SH, feature, uncertainty, in which the loss is
   linear away from the colour clamp), every sample within the same fraction of
   the group's largest gradient, cosine >= 0.999.
"""
import math

import numpy as np
import pytest
import torch

from paper_2311_18482_gb300 import synth
from parity import rel_err, to_np

pytestmark = pytest.mark.gpu

FIELDS = ("means", "log_scales", "quats", "opacity_raw", "sh")
DEC = ("W1", "b1", "W2", "b2", "W3", "b3")


def _t(a, dtype=np.float32):
    return torch.from_numpy(np.ascontiguousarray(a, dtype)).cuda()


def fro(got, ref):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    return float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-30))


@pytest.fixture(scope="module")
def c2():
    return synth.config("c2")


def _render(leg, g, cam):
    proj = leg.le_preprocess(g, cam)
    ids, ranges, K, img = leg.le_bin_render_fwd(cam, proj)
    return proj, ids, ranges, K, img


def test_c2_training_step_crop(leg, orc, c2):
    import paper_2311_18482_gb300 as L
    sc, cam, dec = c2["scene"], c2["camera"], c2["decoder"]
    W, H = cam.W, cam.H
    P = W * H
    assert (sc.N, W, H, dec.W3.shape[0]) == (100_000, 640, 480, 128)
    g = leg.Gaussians.from_scene(sc)
    proj, ids, ranges, K, img = _render(leg, g, cam)
    tgt, rgb_t = c2["target_idx"], c2["rgb_target"]
    loss = torch.zeros(1, device="cuda")
    d_rgb = torch.empty((3, H, W), device="cuda")
    leg.le_rgb_l1(img.rgb, _t(rgb_t), loss, d_rgb)
    out = L.le_decode(L.UNFUSED_FP32, img.feat.view(8, P), tuple(_t(getattr(dec, k)) for k in DEC),
                      unc=img.unc.view(P), target=_t(tgt, np.int32))
    torch.cuda.synchronize()

    # the oracle on the 64x64 centre crop, from brute-force tile lists
    kp = orc.keypath(sc, cam)
    assert K == orc.bin_count(kp)
    pr = orc.project(sc, cam, kp["tiles"])
    x0, y0 = (W // 2 - 32) // 16 * 16, (H // 2 - 32) // 16 * 16
    win = (x0, y0, x0 + 64, y0 + 64)
    tl = [(tx, ty) for ty in range(y0 // 16, y0 // 16 + 4) for tx in range(x0 // 16, x0 // 16 + 4)]
    vals, rr = orc.lists_for_tiles(cam, kp, tl)
    ref = orc.render(cam, sc, pr, vals, rr, win)
    sub = lambda a: a[..., y0:y0 + 64, x0:x0 + 64]
    ok = ref["flip"] == 0
    assert ok.mean() > 0.95            # 98.6 % at this crop
    for k in ("rgb", "feat"):
        assert rel_err(sub(to_np(getattr(img, k)))[:, ok], ref[k][:, ok]) < 1e-4, k
    assert rel_err(sub(to_np(img.unc))[ok], ref["unc"][ok]) < 1e-4
    assert rel_err(sub(to_np(img.T))[ok], ref["T"][ok]) < 1e-4
    assert np.array_equal(sub(to_np(img.n_contrib))[ok], ref["n_contrib"][ok])

    # the oracle's losses over the crop, weighted as the full view's (mean over P pixels)
    tg = sub(rgb_t).astype(np.float64)
    ok &= np.all(np.abs(ref["rgb"] - tg) > 1e-5, axis=0)
    s = 64 * 64 / P
    _, d_rgb_o = orc.l1(ref["rgb"], tg)
    d_rgb_o = d_rgb_o * s
    dl = orc.decoder_loss(ref["feat"].reshape(8, -1), ref["unc"].reshape(-1), sub(tgt).reshape(-1), dec,
                          lambda_ce=s, lambda_u=s)
    d_feat_o = dl["d_feat"].reshape(8, 64, 64)
    d_unc_o = dl["d_unc"].reshape(64, 64)
    g_rgb, g_feat, g_unc = sub(to_np(d_rgb)), sub(to_np(out["d_feat"]).reshape(8, H, W)), \
        sub(to_np(out["d_unc"]).reshape(H, W))
    assert rel_err(g_rgb[:, ok], d_rgb_o[:, ok]) < 1e-4
    assert rel_err(g_feat[:, ok], d_feat_o[:, ok]) < 1e-4
    assert rel_err(g_unc[ok], d_unc_o[ok]) < 1e-4

    # backward from the GPU's own upstream gradients, kept on the crop's valid pixels
    mask = np.zeros((H, W), bool)
    mask[y0:y0 + 64, x0:x0 + 64] = ok
    mk = torch.from_numpy(mask).cuda()
    grads, grad2d = leg.le_render_bwd(cam, g, proj, ids, ranges, img, d_rgb * mk,
                                      out["d_feat"].view(8, H, W) * mk, out["d_unc"].view(H, W) * mk)
    torch.cuda.synchronize()
    z = lambda a, k: np.where(ok, a, 0.0) if a.ndim == 2 else np.where(ok[None], a, 0.0)
    g2 = orc.render_bwd(cam, sc, pr, vals, rr, z(d_rgb_o, 0), z(d_feat_o, 0), z(d_unc_o, 0), window=win)
    gp = orc.project_bwd(sc, cam, kp["tiles"], g2["mean2d"], g2["conic"], g2["opacity"], g2["rgb"])
    for k in FIELDS:
        assert rel_err(to_np(getattr(grads, k)), gp[k]) < 1e-4, k
    assert rel_err(to_np(grads.feat), g2["feat"]) < 1e-4
    assert rel_err(to_np(grads.unc), g2["unc"]) < 1e-4


def test_c2_fused_vs_unfused_whole_view(leg, c2):
    import paper_2311_18482_gb300 as L
    sc, cam, dec = c2["scene"], c2["camera"], c2["decoder"]
    W, H = cam.W, cam.H
    P = W * H
    g = leg.Gaussians.from_scene(sc)
    proj, ids, ranges, K, img = _render(leg, g, cam)
    dec_t = tuple(_t(getattr(dec, k)) for k in DEC)
    tgt = _t(c2["target_idx"], np.int32)
    res = {}
    for name, mode in (("fused", L.FUSED_BF16), ("unfused", L.UNFUSED_FP32)):
        out = L.le_decode(mode, img.feat.view(8, P), dec_t, unc=img.unc.view(P), target=tgt)
        d_rgb = torch.zeros((3, H, W), device="cuda")
        grads, _ = leg.le_render_bwd(cam, g, proj, ids, ranges, img, d_rgb, out["d_feat"].view(8, H, W),
                                     out["d_unc"].view(H, W))
        torch.cuda.synchronize()
        res[name] = (out, {k: to_np(getattr(grads, k)).copy() for k in FIELDS + ("feat", "unc")})
    L.le_device_status()
    (fo, fg), (uo, ug) = res["fused"], res["unfused"]
    errs = {"loss": fro(to_np(fo["loss"]), to_np(uo["loss"])), "d_unc": fro(to_np(fo["d_unc"]), to_np(uo["d_unc"])),
            "d_feat": fro(to_np(fo["d_feat"]), to_np(uo["d_feat"]))}
    for k, gf, gu in zip(DEC, fo["dW"], uo["dW"]):
        errs[k] = fro(to_np(gf), to_np(gu))
    for k in fg:
        errs["grad_" + k] = fro(fg[k], ug[k])
    print("c2 fused vs unfused (relative Frobenius):", {k: f"{v:.2e}" for k, v in errs.items()})
    bars = {"loss": 1e-4, "d_unc": 1e-3, "W3": 2e-2, "b3": 2e-2, "W2": 8e-2, "b2": 8e-2, "W1": 1e-1, "b1": 1e-1,
            "d_feat": 1e-1}
    for k, b in bars.items():
        assert errs[k] <= b, (k, errs[k])
    for k in fg:
        assert errs["grad_" + k] <= 1e-1, (k, errs["grad_" + k])


def test_c2_trained_decoder_on_rendered_features(leg, orc, c2):
    import paper_2311_18482_gb300 as L
    from paper_2311_18482_gb300.training import TrainState
    sc, cam, dec = c2["scene"], c2["camera"], c2["decoder"]
    W, H = cam.W, cam.H
    P = W * H
    st = TrainState(sc, dec, W, H, "cuda", decoder_mode=L.FUSED_BF16)
    tgt_t, rgb_t = _t(c2["target_idx"], np.int32), _t(c2["rgb_target"])
    for _ in range(1000):
        st.step(cam, rgb_t, tgt_t)
    L.le_preprocess(st.g, cam, st.proj)
    L.le_bin_render_fwd(cam, st.proj, st.bins, st.img)
    dec_t = tuple(st.pv[k] for k in DEC)
    am = to_np(L.le_decode(L.FUSED_BF16, st.img.feat.view(8, P), dec_t)["argmax"])
    L.le_device_status()
    f = to_np(st.img.feat).reshape(8, P).astype(np.float64)
    trained = synth.Decoder(*(to_np(st.pv[k]).copy() for k in DEC))
    z = orc.decoder_fwd(f, trained)
    _, am64 = orc.softmax_argmax(z)
    agree = float(np.mean(am == am64))
    diff = np.nonzero(am != am64)[0]
    gap = float(np.max(z[am64[diff], diff] - z[am[diff], diff])) if diff.size else 0.0
    t = c2["target_idx"].reshape(-1)
    cls = np.unique(t)
    means = np.stack([f[:, t == k].mean(1) for k in cls])
    d2 = ((f.T[:, None, :] - means[None]) ** 2).sum(-1)
    nearest = cls[np.argmin(d2, 1)]
    acc, acc_nm = float(np.mean(am == t)), float(np.mean(nearest == t))
    print(f"c2 trained decoder on the rendered view: fused/FP64 argmax agreement {agree:.5f} ({diff.size} pixels, "
          f"largest FP64 logit gap among them {gap:.3f}); accuracy trained {acc:.4f} vs nearest class mean "
          f"{acc_nm:.4f}; losses {to_np(st.loss)}")
    assert agree >= 0.999
    assert gap <= 0.5
    assert acc >= acc_nm + 0.03 and (1 - acc) <= (1 - acc_nm) / 5


def _smooth_fields(rng, n, H, W):
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    out = np.empty((n, H, W))
    for c in range(n):
        f = np.full((H, W), rng.standard_normal())
        for _ in range(3):
            kx, ky = rng.uniform(-3, 3, 2) * 2 * math.pi
            f += 0.5 * np.sin(kx * xx / W + ky * yy / H + rng.uniform(0, 2 * math.pi))
        out[c] = f
    return out


def test_c3_finite_differences_on_gpu(leg):
    c = synth.config("c3")
    sc, cam = c["scene"], c["camera"]
    W, H, N = cam.W, cam.H, sc.N
    rng = np.random.default_rng(9)
    wr, wf, wu = (torch.from_numpy(_smooth_fields(rng, n, H, W)).cuda() for n in (3, 8, 1))
    wu = wu[0]
    g = leg.Gaussians.from_scene(sc)
    proj = leg.le_preprocess(g, cam)
    ids, ranges, K, img = leg.le_bin_render_fwd(cam, proj)
    grads, _ = leg.le_render_bwd(cam, g, proj, ids, ranges, img, wr.float(), wf.float(), wu.float())
    torch.cuda.synchronize()
    reach = np.nonzero(to_np(grads.opacity_raw) != 0)[0]      # Gaussians that reach at least one pixel
    pick = rng.choice(reach, 64, replace=False)
    rec = proj.splat.clone()
    ys, xs = torch.meshgrid(torch.arange(H, device="cuda", dtype=torch.float32),
                            torch.arange(W, device="cuda", dtype=torch.float32), indexing="ij")

    def mask(i):
        """0 where Gaussian i's alpha < 2/255, 1 above 4/255 (the record's base-2 conic)."""
        r = rec[i]
        dx, dy = r[0] - xs, r[1] - ys
        q = r[2] * dx * dx + r[3] * dx * dy + r[4] * dy * dy
        alpha = torch.clamp(r[5] * torch.exp2(-q), max=0.99)
        return torch.clamp((255.0 * alpha.double() - 2.0) / 2.0, 0.0, 1.0)

    proj2 = leg.Projected.empty(N)
    bins = leg.BinSortBuffers()
    img2 = leg.Image.empty(H, W)

    def loss(mr, mf, mu):
        leg.le_preprocess(g, cam, proj2)
        leg.le_bin_render_fwd(cam, proj2, bins, img2)
        return float((img2.rgb.double() * mr).sum() + (img2.feat.double() * mf).sum() +
                     (img2.unc.double() * mu).sum())

    R = np.asarray(cam.view, np.float64).reshape(3, 4)[:, :3]
    groups = {"means": 1e-4, "log_scales": 1e-4, "quats": 1e-4, "opacity_raw": 3e-4, "sh": 1e-2, "feat": 1e-2,
              "unc": 1e-2}
    res = {k: [] for k in groups}
    for i in pick:
        m = mask(i)
        mr, mf, mu = wr * m, wf * m, wu * m
        gi, _ = leg.le_render_bwd(cam, g, proj, ids, ranges, img, mr.float(), mf.float(), mu.float())
        for k, h in groups.items():
            p = getattr(g, k)
            a = getattr(gi, k)[i].double().cpu().numpy().reshape(-1)
            if k == "means":       # in the image plane: the depth order of the lists stays the same
                ab = rng.standard_normal(2)
                v = (ab[0] * R[0] + ab[1] * R[1]) / np.linalg.norm(ab)
            else:
                v = rng.standard_normal(a.size)
                v /= np.linalg.norm(v)
            orig = p[i].clone()
            vt = torch.from_numpy(v.reshape(orig.shape).astype(np.float32)).cuda()
            pp, pm = orig + h * vt, orig - h * vt
            p[i] = pp
            lp = loss(mr, mf, mu)
            p[i] = pm
            lm = loss(mr, mf, mu)
            p[i] = orig
            delta = (pp.double() - pm.double()).cpu().numpy().reshape(-1)   # the FP32 step actually taken
            res[k].append((float(a @ delta), lp - lm))
    print(f"c3 GPU central differences, 64 Gaussians (of {reach.size} that reach a pixel), K = {K}:")
    bad = []
    for k, v in res.items():
        v = np.array(v)
        an, fd = v[:, 0], v[:, 1]
        scale = np.abs(an).max()
        l2 = float(np.linalg.norm(fd - an) / np.linalg.norm(an))
        cos = float(an @ fd / (np.linalg.norm(an) * np.linalg.norm(fd)))
        worst = float(np.abs(fd - an).max() / scale)
        print(f"  {k:12s} relative L2 {l2:.2e} cosine {cos:.6f} worst |fd - an| / max|an| {worst:.2e}")
        bar = 1e-3 if k in ("sh", "feat", "unc") else 2e-2
        if not (scale > 0 and l2 <= bar and worst <= bar and cos >= 0.999):
            bad.append(k)
    assert not bad, bad
