"""GPU parity of the language feature map export (le_feature_map, supp. Sec.
"Inference": F = M_infer S) in BF16.

Two references:
  1. the fused kernel's arithmetic emulated in numpy (BF16 decoder operands,
     e = exp(z - max z) rounded to BF16, codebook rounded to BF16, FP64
     accumulation, 1/sum e of the unrounded e, BF16 output): relative Frobenius
     error <= 3e-3 (the output's own BF16 rounding, 2^-9, and rare 1-ulp flips
     from FP32 accumulation order);
  2. the FP64 oracle F = softmax(D_MLP(R_s)) S: relative Frobenius <= 2e-2 --
     the decoder's BF16 logits move p by <= 1e-2 absolute (the fused decoder's
     bar), and the BF16 roundings of e, S and F add 3 x 2^-9.
"""
import numpy as np
import pytest
import torch

from paper_2311_18482_gb300 import synth
from test_decoder_tc_gpu import _dec_t, _inputs, _t, bf16, emulate_logits, fro

pytestmark = pytest.mark.gpu


# 25,000 pixels are 196 tiles on at most 152 CTAs, so some CTAs run two tiles: with 256 and 240 codes the
# output staging borrows W3's shared memory and W3 is reloaded between a CTA's tiles; with 192 codes the
# staging has its own region (one pair of codebook slots).  With 128 codes or fewer there are two slot
# pairs and the copies run a round ahead, across a CTA's tiles: 7 rounds per tile (896 dims), 2 rounds
# with a one-chunk last round (192 dims), one round per tile (64 dims, copies two tiles ahead).
@pytest.mark.parametrize("P,ncb,d", [(5000, 256, 896), (131, 128, 896), (1, 64, 128), (3000, 16, 192),
                                     (25000, 256, 896), (25000, 240, 896), (25000, 192, 896),
                                     (25000, 128, 896), (25000, 64, 192), (60000, 16, 64)])
def test_feature_map(leg, orc, P, ncb, d):
    import paper_2311_18482_gb300 as L
    dec = synth.decoder_init(31, ncb)
    feat, _, _ = _inputs(P, ncb, 32)
    S = np.random.default_rng(33).standard_normal((ncb, d)).astype(np.float32)
    F = L.le_feature_map(_t(feat), _dec_t(dec), _t(S))
    L.le_device_status()
    got = F.to(torch.float32).cpu().numpy().astype(np.float64)
    z = emulate_logits(feat, dec)
    e = np.exp(z - z.max(0))
    emu = bf16(((bf16(e).T @ bf16(S)) / e.sum(0)[:, None]))
    prob, _ = orc.softmax_argmax(orc.decoder_fwd(feat, dec))
    ref = orc.feature_map(prob, S)
    e1, e2 = fro(got, emu), fro(got, ref)
    print(f"feature map P={P} ncb={ncb} d={d}: vs emulation {e1:.2e}, vs FP64 {e2:.2e}")
    assert e1 <= 3e-3
    assert e2 <= 2e-2


def test_feature_map_one_hot(leg, orc):
    """A decoder whose logits single out one code by a wide margin: F is that code's BF16 row."""
    import paper_2311_18482_gb300 as L
    ncb, P, d = 64, 1000, 896
    dec = synth.decoder_init(34, ncb)
    dec.W3[:] = 0.0
    dec.b3[:] = 0.0
    dec.b3[17] = 60.0          # p = e^-60-close to one-hot on code 17 for every pixel
    feat, _, _ = _inputs(P, ncb, 35)
    S = np.random.default_rng(36).standard_normal((ncb, d)).astype(np.float32)
    F = L.le_feature_map(_t(feat), _dec_t(dec), _t(S))
    torch.cuda.synchronize()
    got = F.to(torch.float32).cpu().numpy()
    assert np.array_equal(got, np.broadcast_to(bf16(S[17]).astype(np.float32), got.shape))


@pytest.mark.parametrize("ncb", [256, 128])
def test_feature_map_full_view_sampled(leg, orc, ncb):
    """The full 1296 x 840 view with 256 codes (every CTA runs ~57 tiles, W3 reloaded between them) and
    with 128 codes (two codebook slot pairs, copies a round ahead) x 896 dims: 1,024 sampled pixels (and
    the last one) against the emulation and the FP64 oracle, row by row."""
    import paper_2311_18482_gb300 as L
    d, P = 896, 1296 * 840
    dec = synth.decoder_init(37, ncb)
    feat, _, _ = _inputs(P, ncb, 38)
    S = np.random.default_rng(39).standard_normal((ncb, d)).astype(np.float32)
    F = L.le_feature_map(_t(feat), _dec_t(dec), _t(S))
    L.le_device_status()
    idx = np.sort(np.concatenate([np.random.default_rng(40).choice(P - 1, 1024, replace=False), [P - 1]]))
    got = F[torch.from_numpy(idx).cuda()].to(torch.float32).cpu().numpy().astype(np.float64)
    del F
    fs = np.ascontiguousarray(feat[:, idx])
    z = emulate_logits(fs, dec)
    e = np.exp(z - z.max(0))
    emu = bf16(((bf16(e).T @ bf16(S)) / e.sum(0)[:, None]))
    prob, _ = orc.softmax_argmax(orc.decoder_fwd(fs, dec))
    ref = orc.feature_map(prob, S)
    e1, e2 = fro(got, emu), fro(got, ref)
    rows = np.linalg.norm(got - emu, axis=1) / np.linalg.norm(emu, axis=1)
    print(f"feature map full view, {len(idx)} sampled pixels: vs emulation {e1:.2e} (worst row {rows.max():.2e}), "
          f"vs FP64 {e2:.2e}")
    assert e1 <= 3e-3 and rows.max() <= 1e-2
    assert e2 <= 2e-2
