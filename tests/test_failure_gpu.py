"""Failure detection and resume on the GPU, without faulting it.

1. A kernel waits on a barrier nothing completes; its bounded wait expires, it
   records the timeout and returns; le_device_status reports LE_ERR_TIMEOUT once
   and the context keeps working (a fused decode afterwards is correct).
2. Checkpoint / resume: a training run restored from a snapshot continues like
   the uninterrupted run (within the order noise of the gradient atomics).
"""
import numpy as np
import pytest
import torch

from paper_2311_18482_gb300 import synth

pytestmark = pytest.mark.gpu


def test_bounded_wait_timeout_is_reported(leg):
    import paper_2311_18482_gb300 as L
    L.le_device_status()                      # clean slate
    L.le_selftest_bounded_wait()
    with pytest.raises(L.LegError) as e:
        L.le_device_status()
    assert e.value.status == L.LE_ERR_TIMEOUT
    L.le_device_status()                      # the record was cleared
    dec = synth.decoder_init(41, 64)
    f = np.random.default_rng(0).standard_normal((8, 500)).astype(np.float32)
    dt = tuple(torch.from_numpy(getattr(dec, k)).cuda() for k in ("W1", "b1", "W2", "b2", "W3", "b3"))
    a = L.le_decode(L.FUSED_BF16, torch.from_numpy(f).cuda(), dt)["argmax"]
    b = L.le_decode(L.UNFUSED_FP32, torch.from_numpy(f).cuda(), dt)["argmax"]
    L.le_device_status()
    assert float((a == b).float().mean()) > 0.98


def test_checkpoint_resume(leg):
    from paper_2311_18482_gb300.training import TrainState
    import paper_2311_18482_gb300 as L
    c = synth.config("c5", n=20000, W=256, H=160)
    sc, dec = c["scene"], c["decoder"]
    views = [(synth.circle_pose(k, 16, 256, 160), torch.from_numpy(synth.smooth_rgb_target(2000 + k, 256, 160)).cuda(),
              torch.from_numpy(synth.voronoi_index_map(1000 + k, 256, 160, 128)).cuda()) for k in range(5)]
    a = TrainState(sc, dec, 256, 160, decoder_mode=L.FUSED_BF16)
    for k in range(3):
        a.step(*views[k])
    snap = a.state_dict()
    for k in range(3, 5):
        a.step(*views[k])
    b = TrainState(sc, dec, 256, 160, decoder_mode=L.FUSED_BF16)
    b.load_state_dict(snap)
    for k in range(3, 5):
        b.step(*views[k])
    torch.cuda.synchronize()
    assert b.step_count == a.step_count == 5
    diff = (a.params - b.params).abs().max().item()
    moved = (a.params - snap["params"].cuda()).abs().max().item()
    assert moved > 1e-4 and diff < 1e-3 * moved
