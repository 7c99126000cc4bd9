"""GPU parity of the semantic decoder (inference and training step) and the
relevancy query against the FP64 oracle, through the C ABI.

Unfused FP32 path: logits / prob / loss within 1e-5 relative, gradients
within 1e-4 relative (per-tensor infinity norm), relevancy within 1e-5
absolute, argmax exact wherever the oracle's top-2 logit gap exceeds 1e-4.
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


def _inputs(P, ncb, seed):
    rng = np.random.default_rng(seed)
    feat = rng.standard_normal((8, P)).astype(np.float32)
    unc = rng.uniform(0, 1, P).astype(np.float32)
    tgt = rng.integers(0, ncb, P).astype(np.int32)
    return feat, unc, tgt


def _clear_top2(logits, tol=1e-4):
    s = np.sort(logits, axis=0)
    return (s[-1] - s[-2]) > tol


@pytest.mark.parametrize("P,ncb", [(3001, 128), (4096, 256), (1, 16)])
def test_decode_inference_unfused(leg, orc, P, ncb):
    import paper_2311_18482_gb300 as L
    dec = synth.decoder_init(5, ncb)
    feat, _, _ = _inputs(P, ncb, 1)
    out = L.le_decode(L.UNFUSED_FP32, _t(feat), _dec_t(dec), want_prob=True, want_logits=True)
    torch.cuda.synchronize()
    z = orc.decoder_fwd(feat, dec)
    prob, am = orc.softmax_argmax(z)
    assert rel_err(to_np(out["logits"]), z) < 1e-5
    assert rel_err(to_np(out["prob"]), prob) < 1e-5
    clear = _clear_top2(z)
    assert np.array_equal(to_np(out["argmax"])[clear], am[clear])


@pytest.mark.parametrize("P,ncb", [(3001, 128), (2048, 64)])
def test_decode_train_unfused(leg, orc, P, ncb):
    import paper_2311_18482_gb300 as L
    dec = synth.decoder_init(6, ncb)
    feat, unc, tgt = _inputs(P, ncb, 2)
    lce, lu = 1.0, 0.5
    out = L.le_decode(L.UNFUSED_FP32, _t(feat), _dec_t(dec), unc=_t(unc), target=_t(tgt, np.int32),
                      lambda_ce=lce, lambda_u=lu)
    torch.cuda.synchronize()
    ref = orc.decoder_loss(feat, unc, tgt, dec, lce, lu)
    assert rel_err(to_np(out["loss"]), ref["loss"]) < 1e-5
    assert rel_err(to_np(out["d_feat"]), ref["d_feat"]) < 1e-4
    assert rel_err(to_np(out["d_unc"]), ref["d_unc"]) < 1e-4
    for k, g in zip(("W1", "b1", "W2", "b2", "W3", "b3"), out["dW"]):
        assert rel_err(to_np(g), ref["d" + k]) < 1e-4, k


@pytest.mark.parametrize("P", [5000, 70000])
def test_query_unfused(leg, orc, P):
    import paper_2311_18482_gb300 as L
    dec = synth.decoder_init(7, 256)
    qin = synth.query_inputs(8, 256)
    feat, _, _ = _inputs(P, 256, 3)
    out = L.le_decode(L.UNFUSED_FP32, _t(feat), _dec_t(dec), want_prob=True, want_argmax=False)
    rel = L.le_query(L.UNFUSED_FP32, P, _t(qin.codebook), qin.d_clip, _t(qin.text), _t(qin.negs),
                     dec_t=_dec_t(dec), prob=out["prob"])
    torch.cuda.synchronize()
    z = orc.decoder_fwd(feat, dec)
    prob, _ = orc.softmax_argmax(z)
    ref = orc.query(prob, qin)
    assert np.max(np.abs(to_np(rel) - ref)) < 1e-5
