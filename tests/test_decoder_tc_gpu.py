"""GPU parity of the fused tcgen05 BF16 decoder paths.

Arithmetic: every MMA operand is rounded to BF16 (unit roundoff u = 2^-9),
accumulation is FP32 in TMEM; bias, ReLU, softmax and CE are FP32.

Two references:
  1. a numpy emulation of exactly those BF16 roundings (FP64 accumulation):
     the kernel must match it to 2e-3 (per-tensor infinity norm relative to
     the tensor's scale; what remains is FP32 accumulation order), and its
     argmax must equal the emulation's wherever the emulated top-2 gap exceeds
     1e-3 -- this checks that the kernel computes what it claims;
  2. the FP64 oracle, with bars derived from the arithmetic: each BF16
     rounding contributes at most u = 2^-9 relative; a gradient that passes
     through r roundings and a sum with cancellation factor kappa (<= 8 here)
     is within r * u * kappa.  Relative Frobenius bars: loss 1e-4 (FP32 after
     the MMAs), d_unc 1e-3, layer 3 (r = 3) 2e-2, layer 2 (r = 6) 8e-2,
     layer 1 and d_feat (r = 9) 1e-1.  Softmax |dp| <= 1e-2, relevancy
     |drel| <= 1e-2.  Argmax: >= 99.9 % for a decoder trained by these kernels
     (decisive logits); for a random-init decoder, whose logits are nearly tied,
     the agreement is reported and must stay >= 99 %.
"""
import numpy as np
import pytest
import torch

from paper_2311_18482_gb300 import synth
from parity import rel_err, to_np

pytestmark = pytest.mark.gpu


def _t(a, dtype=np.float32):
    return torch.from_numpy(np.ascontiguousarray(a, dtype)).cuda()


def _dec_t(dec):
    return tuple(_t(getattr(dec, k)) for k in ("W1", "b1", "W2", "b2", "W3", "b3"))


def bf16(x):
    return torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def emulate_train(feat, unc, tgt, dec, lce, lu):
    """The fused kernel's arithmetic in numpy: BF16-rounded MMA operands, FP64 accumulation."""
    P = feat.shape[1]
    W1, W2, W3 = bf16(dec.W1), bf16(dec.W2), bf16(dec.W3)
    b1, b2, b3 = (getattr(dec, k).astype(np.float64) for k in ("b1", "b2", "b3"))
    f = bf16(feat)
    h1 = bf16(np.maximum(W1 @ f + b1[:, None], 0))
    h2 = bf16(np.maximum(W2 @ h1 + b2[:, None], 0))
    z = W3 @ h2 + b3[:, None]
    m = z.max(0)
    lse = m + np.log(np.exp(z - m).sum(0))
    ce = lse - z[tgt, np.arange(P)]
    sm = np.exp(z - lse)
    oh = np.zeros_like(z)
    oh[tgt, np.arange(P)] = 1
    dz = bf16(lce * (1 - unc.astype(np.float64)) * (sm - oh))
    dh2 = bf16((W3.T @ dz) * (h2 > 0))
    dh1 = bf16((W2.T @ dh2) * (h1 > 0))
    out = {"loss": np.array([(ce * (1 - unc)).mean(), unc.mean()]), "d_feat": (W1.T @ dh1) / P,
           "d_unc": (lu - lce * ce) / P, "dW3": dz @ h2.T / P, "db3": dz.sum(1) / P, "dW2": dh2 @ h1.T / P,
           "db2": dh2.sum(1) / P, "dW1": dh1 @ f.T / P, "db1": dh1.sum(1) / P}
    return out


def emulate_logits(feat, dec):
    W1, W2, W3 = bf16(dec.W1), bf16(dec.W2), bf16(dec.W3)
    h1 = bf16(np.maximum(W1 @ bf16(feat) + dec.b1[:, None], 0))
    h2 = bf16(np.maximum(W2 @ h1 + dec.b2[:, None], 0))
    return W3 @ h2 + dec.b3[:, None]


def fro(got, ref):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    return float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-30))


def _inputs(P, ncb, seed):
    rng = np.random.default_rng(seed)
    feat = rng.standard_normal((8, P)).astype(np.float32)
    unc = rng.uniform(0, 1, P).astype(np.float32)
    tgt = rng.integers(0, ncb, P).astype(np.int32)
    return feat, unc, tgt


@pytest.mark.parametrize("P,ncb", [(3001, 128), (20000, 256), (130, 16), (1, 64)])
def test_fused_inference(leg, orc, P, ncb):
    import paper_2311_18482_gb300 as L
    dec = synth.decoder_init(21, ncb)
    feat, _, _ = _inputs(P, ncb, 22)
    out = L.le_decode(L.FUSED_BF16, _t(feat), _dec_t(dec), want_prob=True)
    L.le_device_status()
    z = orc.decoder_fwd(feat, dec)
    prob, am = orc.softmax_argmax(z)
    got = to_np(out["argmax"])
    agree = float(np.mean(got == am))
    dp = float(np.max(np.abs(to_np(out["prob"]) - prob)))
    ze = emulate_logits(feat, dec)
    zs = np.sort(ze, axis=0)
    clear = (zs[-1] - zs[-2]) > 1e-3
    print(f"fused inference P={P} ncb={ncb}: FP64 argmax agreement {agree:.5f} (random init); BF16-emulation "
          f"agreement on {clear.mean():.4f} of pixels: {np.mean(got[clear] == np.argmax(ze, 0)[clear]):.5f}; "
          f"max|dp| {dp:.2e}")
    assert np.array_equal(got[clear], np.argmax(ze, 0)[clear])
    assert agree >= 0.99
    assert dp <= 1e-2


@pytest.mark.parametrize("P,ncb", [(3001, 128), (20000, 64), (1500, 16)])
def test_fused_train(leg, orc, P, ncb):
    import paper_2311_18482_gb300 as L
    dec = synth.decoder_init(23, ncb)
    feat, unc, tgt = _inputs(P, ncb, 24)
    lce, lu = 1.0, 0.5
    out = L.le_decode(L.FUSED_BF16, _t(feat), _dec_t(dec), unc=_t(unc), target=_t(tgt, np.int32),
                      lambda_ce=lce, lambda_u=lu)
    L.le_device_status()
    ref = orc.decoder_loss(feat, unc, tgt, dec, lce, lu)
    emu = emulate_train(feat, unc, tgt, dec, lce, lu)
    got = {"loss": to_np(out["loss"]), "d_feat": to_np(out["d_feat"]), "d_unc": to_np(out["d_unc"])}
    for k, g in zip(("W1", "b1", "W2", "b2", "W3", "b3"), out["dW"]):
        got["d" + k] = to_np(g)
    e_emu = {k: rel_err(got[k], emu[k]) for k in got}
    e_ref = {k: fro(got[k], ref[k]) for k in got}
    print(f"fused train P={P} ncb={ncb}: vs BF16 emulation " + ", ".join(f"{k} {v:.1e}" for k, v in e_emu.items()))
    print(f"fused train P={P} ncb={ncb}: vs FP64 oracle (Frobenius) " + ", ".join(f"{k} {v:.1e}" for k, v in e_ref.items()))
    for k, v in e_emu.items():
        assert v <= 2e-3, ("emulation", k, v)
    bars = {"loss": 1e-4, "d_unc": 1e-3, "dW3": 2e-2, "db3": 2e-2, "dW2": 8e-2, "db2": 8e-2, "dW1": 1e-1,
            "db1": 1e-1, "d_feat": 1e-1}
    for k, v in e_ref.items():
        assert v <= bars[k], ("oracle", k, v)


def test_fused_train_matches_unfused(leg):
    """Fused BF16 and unfused FP32 training steps agree (same seeded inputs)."""
    import paper_2311_18482_gb300 as L
    P, ncb = 50000, 128
    dec = synth.decoder_init(25, ncb)
    feat, unc, tgt = _inputs(P, ncb, 26)
    args = dict(unc=_t(unc), target=_t(tgt, np.int32))
    a = L.le_decode(L.FUSED_BF16, _t(feat), _dec_t(dec), **args)
    b = L.le_decode(L.UNFUSED_FP32, _t(feat), _dec_t(dec), **args)
    L.le_device_status()
    assert rel_err(to_np(a["loss"]), to_np(b["loss"])) <= 1e-4
    assert fro(to_np(a["d_feat"]), to_np(b["d_feat"])) <= 1e-1
    for k, ga, gb in zip(("W1", "b1", "W2", "b2", "W3", "b3"), a["dW"], b["dW"]):
        assert fro(to_np(ga), to_np(gb)) <= {"W3": 2e-2, "b3": 2e-2, "W2": 8e-2, "b2": 8e-2}.get(k, 1e-1), k


@pytest.mark.parametrize("P,ncb", [(5000, 256), (70001, 256), (3001, 64), (2000, 192), (30000, 192), (30000, 128)])
def test_fused_query(leg, orc, P, ncb):
    import paper_2311_18482_gb300 as L
    dec = synth.decoder_init(27, ncb)
    qin = synth.query_inputs(28, ncb)
    feat, _, _ = _inputs(P, ncb, 29)
    rel = L.le_query(L.FUSED_BF16, P, _t(qin.codebook), qin.d_clip, _t(qin.text), _t(qin.negs), feat=_t(feat),
                     dec_t=_dec_t(dec))
    L.le_device_status()
    z = orc.decoder_fwd(feat, dec)
    prob, _ = orc.softmax_argmax(z)
    ref = orc.query(prob, qin)
    err = float(np.max(np.abs(to_np(rel) - ref)))
    print(f"fused query P={P} ncb={ncb}: max|drel| {err:.2e}")
    assert err <= 1e-2


def test_fused_query_full_view_sampled(leg, orc):
    """The query at the full 1296 x 840 view (every CTA runs ~57 tiles, each tile's R_s loaded a tile
    ahead): 2,048 sampled pixels and the last one against the FP64 oracle."""
    import paper_2311_18482_gb300 as L
    P = 1296 * 840
    dec = synth.decoder_init(41, 256)
    qin = synth.query_inputs(42, 256)
    feat, _, _ = _inputs(P, 256, 43)
    rel = L.le_query(L.FUSED_BF16, P, _t(qin.codebook), qin.d_clip, _t(qin.text), _t(qin.negs), feat=_t(feat),
                     dec_t=_dec_t(dec))
    L.le_device_status()
    idx = np.sort(np.concatenate([np.random.default_rng(44).choice(P - 1, 2048, replace=False), [P - 1]]))
    got = to_np(rel)[:, idx]
    prob, _ = orc.softmax_argmax(orc.decoder_fwd(np.ascontiguousarray(feat[:, idx]), dec))
    ref = orc.query(prob, qin)
    err = float(np.max(np.abs(got - ref)))
    print(f"fused query full view, {len(idx)} sampled pixels: max|drel| {err:.2e}")
    assert err <= 1e-2


def test_trained_decoder_argmax_and_gain(leg, orc):
    """Train D_MLP with the fused training kernel + le_adam (lr 1e-3, betas (0.9,
    0.999), Sec. 4) on features drawn around one random 8-dim prototype per
    codebook entry; then (1) the fused BF16 argmax agrees with the FP64 oracle's
    on >= 99.9 % of fresh pixels and (2) the trained decoder classifies far
    better than the untrained one (what the learned part gains)."""
    import paper_2311_18482_gb300 as L
    P, ncb, steps = 16384, 64, 400
    proto = np.random.default_rng(31).standard_normal((ncb, 8))

    def batch(seed):
        r = np.random.default_rng(seed)
        t = r.integers(0, ncb, P)
        f = (proto[t] + 0.3 * r.standard_normal((P, 8))).T.astype(np.float32)
        return f, t.astype(np.int32)

    dec0 = synth.decoder_init(32, ncb)
    names = ("W1", "b1", "W2", "b2", "W3", "b3")
    sizes = [getattr(dec0, k).size for k in names]
    flat = torch.from_numpy(np.concatenate([getattr(dec0, k).ravel() for k in names])).cuda()
    grad, m, v = torch.zeros_like(flat), torch.zeros_like(flat), torch.zeros_like(flat)
    views = []
    o = 0
    for k, n in zip(names, sizes):
        views.append((o, n, getattr(dec0, k).shape))
        o += n
    W = lambda buf: tuple(buf[a:a + n].view(*shp) for a, n, shp in views)
    zeros_u = torch.zeros(P, device="cuda")
    for step in range(1, steps + 1):
        f, t = batch(step)
        out = L.le_decode(L.FUSED_BF16, _t(f), W(flat), unc=zeros_u, target=_t(t, np.int32))
        for (a, n, shp), g in zip(views, out["dW"]):
            grad[a:a + n].copy_(g.reshape(-1))
        L.le_adam(flat, grad, m, v, step, lr=1e-3)
    L.le_device_status()
    trained = synth.Decoder(*(to_np(x).astype(np.float32) for x in W(flat)))
    f, t = batch(10_000)
    got = to_np(L.le_decode(L.FUSED_BF16, _t(f), W(flat))["argmax"])
    _, am = orc.softmax_argmax(orc.decoder_fwd(f, trained))
    _, am0 = orc.softmax_argmax(orc.decoder_fwd(f, dec0))
    agree = float(np.mean(got == am))
    acc, acc0 = float(np.mean(am == t)), float(np.mean(am0 == t))
    print(f"trained decoder: fused/FP64 argmax agreement {agree:.5f}; accuracy trained {acc:.3f} vs untrained {acc0:.3f}")
    assert agree >= 0.999
    assert acc >= acc0 + 0.3


@pytest.mark.parametrize("mode_name,P,widths", [("fused", 50001, (64, 128)), ("fused", 129, (64, 128)),
                                                ("unfused", 3001, (64, 128)), ("fused", 3001, (128, 256))])
def test_decode_l1_matches_separate_calls(leg, mode_name, P, widths):
    """le_decode_l1 (the RGB L1 term in the decoder's training pass; at 8-64-128 inside the tensor-core
    kernel, otherwise le_rgb_l1 + le_decode) against le_rgb_l1 followed by le_decode on the same
    inputs: d_img bit for bit, d_feat and d_unc bit for bit (the same kernel per pixel), the losses
    and weight gradients up to the order of their FP32 atomic sums.  The L1 loss is a sum of at most
    2 x 152 x 8 nonnegative partials in either form: two orders of m such terms differ by at most
    2 (m - 1) u of the sum (u = 2^-24)."""
    import paper_2311_18482_gb300 as L
    B = L.binding
    mode = L.FUSED_BF16 if mode_name == "fused" else L.UNFUSED_FP32
    ncb = 128
    dec = synth.decoder_init(31, ncb, h1=widths[0], h2=widths[1])
    feat, unc, tgt = _inputs(P, ncb, 32)
    rng = np.random.default_rng(33)
    img, img_t = _t(rng.uniform(0, 1, (3, P))), _t(rng.uniform(0, 1, (3, P)))
    dec_t = _dec_t(dec)
    ds = B.decoder_struct(*dec_t)
    nb = B.le_decode_workspace(mode | B.DECODE_TRAIN, P, ds)
    outs = []
    for fused_l1 in (True, False):
        o = dict(loss=torch.zeros(2, device="cuda"), d_feat=torch.empty(8, P, device="cuda"),
                 d_unc=torch.empty(P, device="cuda"), dW=[torch.empty_like(x) for x in dec_t],
                 l1=torch.full((1,), 7.0, device="cuda"), d_img=torch.full((3, P), 7.0, device="cuda"),
                 ws=torch.empty(max(nb, 1), dtype=torch.uint8, device="cuda"))
        dg = B.decoder_grads_struct(o["dW"])
        if fused_l1:
            B.le_decode_l1_raw(mode, P, _t(feat), _t(unc), ds, _t(tgt, np.int32), 1.0, 1.0, o["loss"], o["d_feat"],
                               o["d_unc"], dg, img, img_t, o["l1"], o["d_img"], o["ws"])
        else:
            B.le_rgb_l1(img, img_t, o["l1"], o["d_img"])
            B.le_decode_raw(mode, P, _t(feat), _t(unc), ds, _t(tgt, np.int32), 1.0, 1.0, o["loss"], o["d_feat"],
                            o["d_unc"], dg, None, None, None, o["ws"])
        outs.append(o)
    torch.cuda.synchronize()
    L.le_device_status()
    a, b = outs
    assert torch.equal(a["d_img"], b["d_img"])
    assert torch.equal(a["d_feat"], b["d_feat"]) and torch.equal(a["d_unc"], b["d_unc"])
    m = 2 * 152 * 8
    l1 = float(b["l1"][0])
    assert abs(float(a["l1"][0]) - l1) <= 2 * (m - 1) * 2.0 ** -24 * l1
    assert abs(l1 - float(np.abs(to_np(img).astype(np.float64) - to_np(img_t)).mean())) <= 1e-5 * l1
    assert rel_err(to_np(a["loss"]), to_np(b["loss"])) <= 1e-5
    for ga, gb in zip(a["dW"], b["dW"]):
        assert rel_err(to_np(ga), to_np(gb)) <= 1e-5
