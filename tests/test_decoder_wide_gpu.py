"""GPU parity of the decoder at the widths of supp. Tab. dmlp (8 -> 128 -> 256 ->
N; Eq. eq:lem_dec) on the tensor cores (csrc/decoder_wide.cu), through le_decode.

The arithmetic is that of the narrower fused kernels: every MMA operand is
rounded to BF16 (u = 2^-9), accumulation is FP32 in TMEM, bias, ReLU, softmax and
cross-entropy are FP32, and dL/dz is rounded to BF16 before the 1/P scale.  So
the same two references and bars apply (tests/test_decoder_tc_gpu.py):
  1. the numpy emulation of those roundings: every output within 2e-3 of its
     scale, argmax equal wherever the emulated top-2 gap exceeds 1e-3;
  2. the FP64 oracle (orc.decoder_fwd / orc.decoder_loss, whose widths come from
     the weights): softmax |dp| <= 1e-2, argmax agreement >= 99 % for a random
     decoder; relative Frobenius loss 1e-4, d_unc 1e-3, layer 3 2e-2, layer 2
     8e-2, layer 1 and d_feat 1e-1 (r BF16 roundings x kappa <= 8 cancellation).
Cases cover one to several tiles per CTA, 16 to 256 codes (above 128 the codes'
W3 halves take turns in one shared-memory slot, in alternating order per tile),
a ragged last tile, and 300,000 pixels (about 15 tiles per CTA).  A training run with the
kernels' own gradients and Adam checks the >= 99.9 % argmax agreement of a trained
decoder at these widths, and the unfused FP32 path is compared on the same step.
"""
import numpy as np
import pytest
import torch

from paper_2311_18482_gb300 import synth
from parity import rel_err, to_np
from test_decoder_tc_gpu import _dec_t, _inputs, _t, emulate_logits, emulate_train, fro

pytestmark = pytest.mark.gpu


def _wide(seed, ncb):
    return synth.decoder_init(seed, ncb, h1=128, h2=256)


@pytest.mark.parametrize("P,ncb", [(3001, 128), (20000, 256), (130, 16), (1, 64), (40000, 192)])
def test_wide_inference(leg, orc, P, ncb):
    import paper_2311_18482_gb300 as L
    dec = _wide(51, ncb)
    feat, _, _ = _inputs(P, ncb, 52)
    out = L.le_decode(L.FUSED_BF16, _t(feat), _dec_t(dec), want_prob=True)
    L.le_device_status()
    got = to_np(out["argmax"])
    ze = emulate_logits(feat, dec)
    zs = np.sort(ze, axis=0)
    clear = (zs[-1] - zs[-2]) > 1e-3
    pe = np.exp(ze - ze.max(0))
    pe /= pe.sum(0)
    prob = to_np(out["prob"])
    z = orc.decoder_fwd(feat, dec)
    p64, am = orc.softmax_argmax(z)
    agree = float(np.mean(got == am))
    dp = float(np.max(np.abs(prob - p64)))
    print(f"wide inference P={P} ncb={ncb}: emulation argmax on {clear.mean():.4f} of pixels, max|dp| vs emulation "
          f"{np.max(np.abs(prob - pe)):.2e}; FP64 agreement {agree:.5f}, max|dp| {dp:.2e}")
    assert np.array_equal(got[clear], np.argmax(ze, 0)[clear])
    assert np.max(np.abs(prob - pe)) <= 2e-3
    assert agree >= 0.99 and dp <= 1e-2


@pytest.mark.parametrize("P,ncb", [(3001, 128), (20000, 64), (1500, 16), (1, 32), (300000, 128)])
def test_wide_train(leg, orc, P, ncb):
    import paper_2311_18482_gb300 as L
    dec = _wide(53, ncb)
    feat, unc, tgt = _inputs(P, ncb, 54)
    lce, lu = 1.0, 0.5
    out = L.le_decode(L.FUSED_BF16, _t(feat), _dec_t(dec), unc=_t(unc), target=_t(tgt, np.int32),
                      lambda_ce=lce, lambda_u=lu)
    L.le_device_status()
    got = {"loss": to_np(out["loss"]), "d_feat": to_np(out["d_feat"]), "d_unc": to_np(out["d_unc"])}
    for k, g in zip(("W1", "b1", "W2", "b2", "W3", "b3"), out["dW"]):
        got["d" + k] = to_np(g)
    emu = emulate_train(feat, unc, tgt, dec, lce, lu)
    e_emu = {k: rel_err(got[k], emu[k]) for k in got}
    print(f"wide train P={P} ncb={ncb}: vs BF16 emulation " + ", ".join(f"{k} {v:.1e}" for k, v in e_emu.items()))
    for k, v in e_emu.items():
        assert v <= 2e-3, ("emulation", k, v)
    if P <= 20000:
        ref = orc.decoder_loss(feat, unc, tgt, dec, lce, lu)
        e_ref = {k: fro(got[k], ref[k]) for k in got}
        print(f"wide train P={P} ncb={ncb}: vs FP64 oracle (Frobenius) " +
              ", ".join(f"{k} {v:.1e}" for k, v in e_ref.items()))
        bars = {"loss": 1e-4, "d_unc": 1e-3, "dW3": 2e-2, "db3": 2e-2, "dW2": 8e-2, "db2": 8e-2, "dW1": 1e-1,
                "db1": 1e-1, "d_feat": 1e-1}
        for k, v in e_ref.items():
            assert v <= bars[k], ("oracle", k, v)


def test_wide_train_matches_unfused(leg):
    """The tensor-core and the unfused FP32 training steps at these widths agree on the same inputs."""
    import paper_2311_18482_gb300 as L
    P, ncb = 50000, 128
    dec = _wide(55, ncb)
    feat, unc, tgt = _inputs(P, ncb, 56)
    args = dict(unc=_t(unc), target=_t(tgt, np.int32))
    a = L.le_decode(L.FUSED_BF16, _t(feat), _dec_t(dec), **args)
    b = L.le_decode(L.UNFUSED_FP32, _t(feat), _dec_t(dec), **args)
    L.le_device_status()
    assert rel_err(to_np(a["loss"]), to_np(b["loss"])) <= 1e-4
    assert fro(to_np(a["d_feat"]), to_np(b["d_feat"])) <= 1e-1
    for k, ga, gb in zip(("W1", "b1", "W2", "b2", "W3", "b3"), a["dW"], b["dW"]):
        assert fro(to_np(ga), to_np(gb)) <= {"W3": 2e-2, "b3": 2e-2, "W2": 8e-2, "b2": 8e-2}.get(k, 1e-1), k


def test_wide_trained_argmax(leg, orc):
    """Train the 8-128-256-64 decoder with its own tensor-core gradients and Adam (lr 1e-3) on
    features drawn around one 8-dim prototype per code; the fused argmax then agrees with the FP64
    oracle's on >= 99.9 % of fresh pixels, and the trained decoder classifies far better than the
    untrained one."""
    import paper_2311_18482_gb300 as L
    P, ncb, steps = 16384, 64, 300
    proto = np.random.default_rng(57).standard_normal((ncb, 8))

    def batch(seed):
        r = np.random.default_rng(seed)
        t = r.integers(0, ncb, P)
        f = (proto[t] + 0.3 * r.standard_normal((P, 8))).T.astype(np.float32)
        return f, t.astype(np.int32)

    dec0 = _wide(58, ncb)
    names = ("W1", "b1", "W2", "b2", "W3", "b3")
    flat = torch.from_numpy(np.concatenate([getattr(dec0, k).ravel() for k in names])).cuda()
    grad, m, v = torch.zeros_like(flat), torch.zeros_like(flat), torch.zeros_like(flat)
    views, o = [], 0
    for k in names:
        n = getattr(dec0, k).size
        views.append((o, n, getattr(dec0, k).shape))
        o += n
    W = lambda buf: tuple(buf[a:a + n].view(*shp) for a, n, shp in views)
    zeros_u = torch.zeros(P, device="cuda")
    ws = None
    for step in range(1, steps + 1):
        f, t = batch(step)
        out = L.le_decode(L.FUSED_BF16, _t(f), W(flat), unc=zeros_u, target=_t(t, np.int32), workspace=ws)
        ws = out["workspace"]
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
    print(f"wide trained decoder: fused/FP64 argmax agreement {agree:.5f}; accuracy {acc:.3f} vs untrained {acc0:.3f}")
    assert agree >= 0.999
    assert acc >= acc0 + 0.3
