"""GPU parity of the adaptive spatial smoothing (le_smooth, Sec. 3.4) on the
tensor cores.

Two references:
  1. a float32 emulation of the kernel's BF16 rounding points (positions,
     weights, hidden activations, dL/ds_MLP and the hidden gradients rounded to
     BF16; everything else FP32): every output within 2e-3 (relative Frobenius),
     which leaves only the tensor cores' FP32 accumulation order and the rare
     ReLU decision at a pre-activation within rounding of 0;
  2. the FP64 oracle, relative Frobenius: s_MLP and the loss 1e-2, d_feat 2e-2,
     the MLP parameter gradients r u kappa with u = 2^-9 per BF16 rounding, r the
     roundings on the path (layer 4: 3, layer 3: 5, layers 2 and 1: 7 and 9) and
     kappa <= 8 for the cancellation in 128-term sums: 5e-2, 8e-2, 1.1e-1, 1.4e-1.
     Measured at random initialisation: <= 5e-3 (layer 4), <= 7.5e-2 (layers 1-3,
     n = 129; smaller with more Gaussians averaged).
"""
import numpy as np
import pytest
import torch

from paper_2311_18482_gb300 import synth

pytestmark = pytest.mark.gpu

KEYS = ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    mlp = synth.smooth_mlp_init(seed)
    means = rng.uniform(-2, 2, (n, 3)).astype(np.float32)
    feat = rng.standard_normal((n, 8)).astype(np.float32)
    unc = rng.uniform(0, 0.4, n).astype(np.float32)
    return mlp, means, feat, unc


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _bf(x):
    return x.to(torch.bfloat16).to(torch.float32)


def _emulate(mlp, means, feat, unc, w_s, lam):
    t = lambda a: torch.from_numpy(np.asarray(a, np.float32))
    W = {k: t(getattr(mlp, k)) for k in KEYS}
    Wb = {k: _bf(W[k]) for k in ("W1", "W2", "W3", "W4")}
    X = _bf(t(means))
    p1 = X @ Wb["W1"].T + W["b1"]
    H1 = _bf(torch.relu(p1))
    p2 = H1 @ Wb["W2"].T + W["b2"]
    H2 = _bf(torch.relu(p2))
    p3 = H2 @ Wb["W3"].T + W["b3"]
    H3 = _bf(torch.relu(p3))
    z = H3 @ Wb["W4"].T + W["b4"]
    diff = z - t(feat)
    nn = torch.linalg.norm(diff, dim=1)
    n = means.shape[0]
    wgt = torch.clamp(t(unc), min=w_s)
    loss = lam / n * torch.sum((1 + wgt) * nn)
    dz = torch.where(nn[:, None] > 0, diff / nn[:, None], torch.zeros_like(diff)) * (lam / n)
    d_feat = -wgt[:, None] * dz
    dzb = _bf(dz)
    dH3 = _bf((dzb @ Wb["W4"]) * (p3 > 0))
    dH2 = _bf((dH3 @ Wb["W3"]) * (p2 > 0))
    dH1 = _bf((dH2 @ Wb["W2"]) * (p1 > 0))
    g = {"W4": dzb.T @ H3, "b4": dz.sum(0), "W3": dH3.T @ H2, "b3": dH3.sum(0), "W2": dH2.T @ H1,
         "b2": dH2.sum(0), "W1": dH1.T @ X, "b1": dH1.sum(0)}
    return {"s_mlp": z.numpy(), "loss": float(loss), "d_feat": d_feat.numpy(), **{"d" + k: v.numpy() for k, v in g.items()}}


def _run(leg, mlp, means, feat, unc, w_s=0.1, lam=1.0):
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    params = {k: c(getattr(mlp, k)) for k in KEYS}
    loss, d_feat, grads, s_mlp = leg.le_smooth(c(means), c(feat), c(unc), params, w_s=w_s, lambda_smo=lam,
                                               want_s_mlp=True)
    torch.cuda.synchronize()
    out = {"loss": float(loss.item()), "d_feat": d_feat.cpu().numpy(), "s_mlp": s_mlp.cpu().numpy()}
    for k, gk in zip(KEYS, grads):
        out["d" + k] = gk.cpu().numpy()
    return out


@pytest.mark.parametrize("n", [5000, 1, 129, 20000])
def test_smooth_vs_bf16_emulation_and_oracle(leg, orc, n):
    mlp, means, feat, unc = _inputs(n, 70 + n % 13)
    got = _run(leg, mlp, means, feat, unc, lam=0.8)
    emu = _emulate(mlp, means, feat, unc, 0.1, 0.8)
    ref = orc.smooth(means, feat, unc, mlp, w_s=0.1, lam=0.8)
    for k in ("s_mlp", "d_feat") + tuple("d" + k for k in KEYS):
        e = _rel(got[k], emu[k])
        print(f"n={n} {k}: vs BF16 emulation {e:.2e}, vs FP64 {_rel(got[k], ref[k]):.2e}")
        assert e <= 2e-3, (k, e)
    assert abs(got["loss"] - emu["loss"]) <= 2e-3 * abs(emu["loss"])
    assert _rel(got["s_mlp"], ref["s_mlp"]) <= 1e-2
    assert abs(got["loss"] - ref["loss"]) <= 1e-2 * abs(ref["loss"])
    assert _rel(got["d_feat"], ref["d_feat"]) <= 2e-2
    bars = {"W4": 5e-2, "b4": 5e-2, "W3": 8e-2, "b3": 8e-2, "W2": 1.1e-1, "b2": 1.1e-1, "W1": 1.4e-1,
            "b1": 1.4e-1}
    for k in KEYS:
        assert _rel(got["d" + k], ref["d" + k]) <= bars[k], k


# (offset, stride) in floats: grad2d's feature slots (8-byte aligned rows), an odd offset (4-byte
# aligned rows), a 16-byte aligned strided layout
@pytest.mark.parametrize("off,stride", [(10, 20), (9, 20), (12, 24)])
def test_smooth_accumulates_into_strided_records(leg, orc, off, stride):
    """d_feat is added into the feature slots of strided records (grad2d + 10, stride 20, in training)."""
    n = 3000
    mlp, means, feat, unc = _inputs(n, 90)
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    params = {k: c(getattr(mlp, k)) for k in KEYS}
    rec = torch.randn((n, stride), device="cuda")
    before = rec.clone()
    loss, _, grads, _ = leg.le_smooth(c(means), c(feat), c(unc), params, d_feat=rec[:, off:],
                                      d_feat_stride=stride)
    dense = _run(leg, mlp, means, feat, unc)
    torch.cuda.synchronize()
    assert torch.equal(rec[:, :off], before[:, :off]) and torch.equal(rec[:, off + 8:], before[:, off + 8:])
    # rec = before + d_feat element by element (one FP32 rounding of the sum, at most a
    # couple of ulps of `before` away from adding the dense result afterwards)
    expect = before[:, off:off + 8].cpu().numpy().astype(np.float64) + dense["d_feat"]
    got = rec[:, off:off + 8].cpu().numpy().astype(np.float64)
    assert np.abs(got - expect).max() <= 2.5e-7 * np.abs(expect).max()
    assert np.abs(dense["d_feat"]).max() > 1e-5
