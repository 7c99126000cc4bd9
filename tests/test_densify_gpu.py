"""GPU parity of adaptive density control (le_densify_stats, le_densify)
against the oracle: statistics and decisions bit-exact (fixed FP32
operations), copied parameters and moments bit-exact, split children's
means within 1e-6 of the scene scale (FP32 rotation vs FP64) and their
log-scales within 1e-6."""
import numpy as np
import pytest
import torch

from test_oracle_pins import _densify_inputs

pytestmark = pytest.mark.gpu

FIELDS = ("means", "log_scales", "quats", "opacity_raw", "sh", "feat", "unc")


def _gauss(leg, d):
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return leg.Gaussians(*(c(d[k]) for k in FIELDS), 3)


def test_densify_stats_exact(leg, orc):
    rng = np.random.default_rng(80)
    n = 50001
    acc = np.zeros(n, np.float32)
    cnt = np.zeros(n, np.int32)
    acc_t = torch.zeros(n, device="cuda")
    cnt_t = torch.zeros(n, dtype=torch.int32, device="cuda")
    for step in range(3):
        g2 = rng.standard_normal((n, 20)).astype(np.float32) * np.float32(1e-3)
        rad = rng.integers(0, 3, n).astype(np.int32)
        leg.le_densify_stats(torch.from_numpy(g2).cuda(), torch.from_numpy(rad).cuda(), acc_t, cnt_t)
        orc.densify_stats(g2[:, :2], rad, acc, cnt)     # the record's first two floats: dL/dmean2d
    torch.cuda.synchronize()
    assert np.array_equal(acc_t.cpu().numpy().view(np.uint32), acc.view(np.uint32))
    assert np.array_equal(cnt_t.cpu().numpy(), cnt)


@pytest.mark.parametrize("n", [4000, 1025, 1])
def test_densify_matches_oracle(leg, orc, n):
    P, acc, cnt = _densify_inputs(n, 81 + n)
    rng = np.random.default_rng(82)
    M = {k: rng.standard_normal(v.shape).astype(np.float32) for k, v in P.items()}
    V = {k: rng.uniform(0, 1, v.shape).astype(np.float32) for k, v in P.items()}
    noise = rng.standard_normal((n, 2, 3)).astype(np.float32)
    cfg = dict(grad_thresh=0.0002, percent_dense=0.01, min_opacity=0.005)
    gp, gm, gv = leg.le_densify(_gauss(leg, P), _gauss(leg, M), _gauss(leg, V), torch.from_numpy(acc).cuda(),
                                torch.from_numpy(cnt).cuda(), torch.from_numpy(noise).cuda(), scene_extent=4.0, **cfg)
    torch.cuda.synchronize()
    o = orc.densify(P, M, V, acc, cnt, noise, extent=4.0, **cfg)
    assert gp.n == o["n_out"]
    kind = o["kind"]
    nk = int(np.sum((kind == 1) | (kind == 2)) + np.sum(kind == 2))     # kept + clones: exact copies
    for k in FIELDS:
        got = getattr(gp, k).cpu().numpy()
        ref = o["params"][k]
        if k in ("means", "log_scales"):
            assert np.array_equal(got[:nk], ref[:nk].astype(np.float32)), k
            tol = 1e-6 * max(1.0, float(np.abs(ref).max()))
            assert np.abs(got[nk:] - ref[nk:]).max(initial=0.0) <= tol, k
        else:
            assert np.array_equal(got, ref), k
        assert np.array_equal(getattr(gm, k).cpu().numpy(), o["m"][k]), k
        assert np.array_equal(getattr(gv, k).cpu().numpy(), o["v"][k]), k


def test_densify_capacity(leg):
    P, acc, cnt = _densify_inputs(3000, 83)
    noise = torch.zeros((3000, 2, 3), device="cuda")
    with pytest.raises(leg.LegError) as e:
        leg.le_densify(_gauss(leg, P), _gauss(leg, P), _gauss(leg, P), torch.from_numpy(acc).cuda(),
                       torch.from_numpy(cnt).cuda(), noise, scene_extent=4.0, n_cap=10)
    assert e.value.status == leg.LE_ERR_CAPACITY
