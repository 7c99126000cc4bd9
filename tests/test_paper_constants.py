"""The configuration the paper prints (tests/golden/paper_hyperparameters.json, each value
with its passage) against the defaults of the oracle, the seeded inputs and the library's
Python binding: a default that drifted from the paper fails here.  CPU only (no compute)."""
import inspect
import json
import os

import pytest

import oracle
from paper_2311_18482_gb300 import binding as B
from paper_2311_18482_gb300 import synth
from paper_2311_18482_gb300.training import TrainState

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_hyperparameters.json")))


def g(key):
    return GOLD[key]["value"]


def defaults(f):
    return {k: p.default for k, p in inspect.signature(f).parameters.items() if p.default is not inspect._empty}


def test_every_value_is_cited():
    for k, v in GOLD.items():
        if not k.startswith("_"):
            assert v["cite"] and "value" in v, k


def test_semantic_feature_width():
    assert synth.D_FEAT == g("d_s")
    c = synth.config("c1", n=50, W=16, H=16)
    assert c["scene"].feat.shape[1] == g("d_s")


@pytest.mark.parametrize("f", [oracle.quantize, B.le_quantize])
def test_quantisation_weights(f):
    d = defaults(f)
    assert d["lambda_d"] == g("lambda_D")
    assert d["lambda_lb"] == g("lambda_lb")
    assert d["lambda_cos"] == g("lambda_other")


def test_smoothing_weights():
    assert defaults(oracle.smooth)["w_s"] == g("w_S")
    assert defaults(oracle.smooth)["lam"] == g("lambda_other")
    assert defaults(B.le_smooth)["w_s"] == g("w_S")
    assert defaults(B.le_smooth)["lambda_smo"] == g("lambda_other")


@pytest.mark.parametrize("f", [oracle.decoder_loss, B.le_decode])
def test_decoder_loss_weights(f):
    d = defaults(f)
    assert d["lambda_ce"] == g("lambda_other") and d["lambda_u"] == g("lambda_other")


def test_adam_settings():
    do, db = defaults(oracle.adam), defaults(B.le_adam)
    assert do["lr"] == db["lr"] == defaults(TrainState)["lr"] == g("adam_lr")
    assert [do["b1"], do["b2"]] == [db["beta1"], db["beta2"]] == g("adam_betas")


def test_mlp_widths():
    w = synth.smooth_mlp_init(0)
    dims = [getattr(w, f"W{k}").shape for k in range(1, 5)]
    assert [dims[0][1]] + [d[0] for d in dims] == g("smoothing_mlp_widths")
    # the paper-width decoder as the seeded inputs build it (the narrower 8-64-128 default is
    # this implementation's workload reading, checked separately by its own tests)
    d = synth.decoder_init(0, max(g("codebook_sizes")), h1=g("decoder_widths")[1], h2=g("decoder_widths")[2])
    assert [d.W1.shape[1], d.W1.shape[0], d.W2.shape[0]] == g("decoder_widths")
    assert d.W3.shape[0] in g("codebook_sizes")
