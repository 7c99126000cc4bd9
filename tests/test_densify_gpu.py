"""GPU parity of adaptive density control (le_densify_stats, le_densify,
le_opacity_reset) against the oracle: statistics (gradient sums, counts,
largest screen radii) and decisions bit-exact (fixed FP32 operations), with
and without the size pruning; copied parameters and moments bit-exact, split
children's means within 1e-6 of the scene scale (FP32 rotation vs FP64) and
their log-scales within 1e-6; the opacity reset bit-exact."""
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
    mr = np.zeros(n, np.int32)
    acc_t = torch.zeros(n, device="cuda")
    cnt_t = torch.zeros(n, dtype=torch.int32, device="cuda")
    mr_t = torch.zeros(n, dtype=torch.int32, device="cuda")
    for step in range(3):
        g2 = rng.standard_normal((n, 20)).astype(np.float32) * np.float32(1e-3)
        rad = rng.integers(0, 3, n).astype(np.int32) * rng.integers(0, 40, n).astype(np.int32)
        leg.le_densify_stats(torch.from_numpy(g2).cuda(), torch.from_numpy(rad).cuda(), acc_t, cnt_t, mr_t)
        orc.densify_stats(g2[:, :2], rad, acc, cnt, mr)     # the record's first two floats: dL/dmean2d
    torch.cuda.synchronize()
    assert np.array_equal(acc_t.cpu().numpy().view(np.uint32), acc.view(np.uint32))
    assert np.array_equal(cnt_t.cpu().numpy(), cnt)
    assert np.array_equal(mr_t.cpu().numpy(), mr)


@pytest.mark.parametrize("n,size_pruning", [(4000, False), (1025, False), (1, False), (4000, True), (1025, True)])
def test_densify_matches_oracle(leg, orc, n, size_pruning):
    P, acc, cnt = _densify_inputs(n, 81 + n)
    rng = np.random.default_rng(82)
    M = {k: rng.standard_normal(v.shape).astype(np.float32) for k, v in P.items()}
    V = {k: rng.uniform(0, 1, v.shape).astype(np.float32) for k, v in P.items()}
    noise = rng.standard_normal((n, 2, 3)).astype(np.float32)
    cfg = dict(grad_thresh=0.0002, percent_dense=0.01, min_opacity=0.005)
    mr = None
    if size_pruning:
        P["log_scales"] = rng.normal(-1.5, 1.0, (n, 3)).astype(np.float32)
        mr = rng.integers(0, 40, n).astype(np.int32)
        cfg.update(max_screen_size=20.0, world_frac=0.1)
    gp, gm, gv = leg.le_densify(_gauss(leg, P), _gauss(leg, M), _gauss(leg, V), torch.from_numpy(acc).cuda(),
                                torch.from_numpy(cnt).cuda(), torch.from_numpy(noise).cuda(), scene_extent=4.0,
                                max_radius=None if mr is None else torch.from_numpy(mr).cuda(), **cfg)
    torch.cuda.synchronize()
    o = orc.densify(P, M, V, acc, cnt, noise, extent=4.0, max_radius=mr, **cfg)
    assert gp.n == o["n_out"]
    if size_pruning and n > 1:
        assert np.sum(o["kind"] == 0) > np.sum(P["opacity_raw"] < orc.densify_thresholds(0, 0.01, 4.0, 0.005)[2])
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


def test_opacity_reset_exact(leg, orc):
    rng = np.random.default_rng(84)
    raw = rng.normal(0, 4, 10007).astype(np.float32)
    m = rng.standard_normal(raw.size).astype(np.float32)
    v = rng.uniform(0, 1, raw.size).astype(np.float32)
    t = [torch.from_numpy(a.copy()).cuda() for a in (raw, m, v)]
    leg.le_opacity_reset(*t, max_opacity=0.01)
    torch.cuda.synchronize()
    orc.opacity_reset(raw, m, v, 0.01)
    for got, want in zip(t, (raw, m, v)):
        assert np.array_equal(got.cpu().numpy().view(np.uint32), want.view(np.uint32))
    with pytest.raises(leg.LegError):
        leg.le_opacity_reset(*t, max_opacity=1.5)
