"""Pins for the FP64 oracle: closed forms, invariants, library special cases,
brute force and finite differences.  CPU only (no GPU, no CUDA library).

Each test pins one oracle function to something other than itself, so that a
dropped term, a wrong sign or index or a transposed operand fails here.
"""
import math

import numpy as np
import pytest

from paper_2311_18482_gb300 import synth

Y00 = 0.5 / math.sqrt(math.pi)         # textbook l=0 real spherical harmonic


def ident_camera(W=32, H=32, f=100.0, bg=(0.0, 0.0, 0.0)):
    view = np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], np.float32)
    return synth.Camera(view=view, campos=np.zeros(3, np.float32), fx=f, fy=f, cx=(W - 1) / 2, cy=(H - 1) / 2,
                        W=W, H=H, bg=np.asarray(bg, np.float32))


def tiny_scene(means, log_scales, quats=None, opacity=None, rgb=None, feat=None, unc=None):
    n = len(means)
    means = np.asarray(means, np.float32).reshape(n, 3)
    log_scales = np.asarray(log_scales, np.float32).reshape(n, 3)
    quats = np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)) if quats is None else np.asarray(quats, np.float32)
    o = np.full(n, 0.5) if opacity is None else np.asarray(opacity, np.float64)
    opacity_raw = np.log(o / (1 - o)).astype(np.float32)
    rgb = np.full((n, 3), 0.5) if rgb is None else np.asarray(rgb, np.float64)
    sh = ((rgb - 0.5) / Y00).astype(np.float32).reshape(n, 1, 3)
    feat = np.zeros((n, 8), np.float32) if feat is None else np.asarray(feat, np.float32)
    unc = np.zeros(n, np.float32) if unc is None else np.asarray(unc, np.float32)
    return synth.Scene(means, log_scales, quats, opacity_raw, sh, feat, unc, 0)


# --------------------------------------------------------------------------- exp
def test_exp_f32_accuracy(orc):
    xs = np.concatenate([np.linspace(-20, 20, 20001), np.random.default_rng(0).normal(-3, 0.5, 5000)])
    xs = xs.astype(np.float32)
    got = np.array([orc.exp_f32(float(x)) for x in xs], np.float64)
    ref = np.exp(xs.astype(np.float64))
    assert np.max(np.abs(got / ref - 1)) < 2.5e-7


# --------------------------------------------------------------------------- SH
def _real_sh_scipy(l, m, d):
    from scipy import special
    theta = math.acos(max(-1.0, min(1.0, d[2])))
    phi = math.atan2(d[1], d[0])
    am = abs(m)
    if hasattr(special, "sph_harm_y"):
        Ylm = complex(special.sph_harm_y(l, am, theta, phi))
    else:
        Ylm = complex(special.sph_harm(am, l, phi, theta))
    if m == 0:
        return Ylm.real
    return math.sqrt(2) * (Ylm.real if m > 0 else Ylm.imag)


def test_sh_matches_scipy(orc):
    rng = np.random.default_rng(1)
    for _ in range(50):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        Y, _ = orc.sh_basis(3, d)
        for l in range(4):
            for m in range(-l, l + 1):
                assert abs(Y[l * l + l + m] - _real_sh_scipy(l, m, d)) < 1e-12, (l, m)


def test_sh_orthonormal(orc):
    x, w = np.polynomial.legendre.leggauss(12)
    nphi = 24
    G = np.zeros((16, 16))
    for ct, wt in zip(x, w):
        st = math.sqrt(1 - ct * ct)
        for k in range(nphi):
            ph = 2 * math.pi * k / nphi
            d = np.array([st * math.cos(ph), st * math.sin(ph), ct])
            Y, _ = orc.sh_basis(3, d)
            G += np.outer(Y, Y) * wt * (2 * math.pi / nphi)
    assert np.max(np.abs(G - np.eye(16))) < 1e-12


def test_sh_tangent_gradient(orc):
    rng = np.random.default_rng(2)
    for _ in range(20):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        t = rng.standard_normal(3)
        t -= d * (d @ t)
        t /= np.linalg.norm(t)
        _, dY = orc.sh_basis(3, d)
        h = 1e-6
        yp, _ = orc.sh_basis(3, (d + h * t) / np.linalg.norm(d + h * t))
        ym, _ = orc.sh_basis(3, (d - h * t) / np.linalg.norm(d - h * t))
        assert np.max(np.abs((yp - ym) / (2 * h) - dY @ t)) < 1e-7


# --------------------------------------------------------------------------- projection
def test_single_isotropic_gaussian_conic(orc):
    f, z, s = 100.0, 4.0, 0.05
    cam = ident_camera(f=f)
    sc = tiny_scene([[0, 0, z]], [[math.log(s)] * 3])
    s = math.exp(float(sc.log_scales[0, 0]))          # the FP32-stored scale
    kp = orc.keypath(sc, cam)
    pr = orc.project(sc, cam, kp["tiles"])
    a = (f * s / z) ** 2 + 0.3
    np.testing.assert_allclose(pr["cov2d"][0], [a, 0, a], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(pr["conic"][0], [1 / a, 0, 1 / a], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(pr["mean2d"][0], [cam.cx, cam.cy], atol=1e-12)
    assert pr["depth"][0] == z
    r = math.ceil(3 * math.sqrt(a))
    assert kp["radius"][0] == r
    # screen mean 15.5 +- r: tiles [floor((15.5-r)/16), floor((15.5+r+15)/16)) clamped to [0,2)
    lo = max(0, math.floor((15.5 - r) / 16))
    hi = min(2, math.floor((15.5 + r + 15) / 16))
    assert list(kp["rect"][0]) == [lo, lo, hi, hi]
    np.testing.assert_allclose(kp["cov2d"][0], [a, 0, a], rtol=1e-6)


def test_anisotropic_axis_aligned_and_rotated(orc):
    f, z = 100.0, 5.0
    s = (0.08, 0.02, 0.05)
    cam = ident_camera(f=f)
    q90 = [math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)]
    sc = tiny_scene([[0, 0, z], [0, 0, z]], [[math.log(v) for v in s]] * 2, quats=[[1, 0, 0, 0], q90])
    s = np.exp(sc.log_scales[0].astype(np.float64))
    kp = orc.keypath(sc, cam)
    pr = orc.project(sc, cam, kp["tiles"])
    a = (f * s[0] / z) ** 2 + 0.3
    c = (f * s[1] / z) ** 2 + 0.3
    np.testing.assert_allclose(pr["cov2d"][0], [a, 0, c], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(pr["cov2d"][1], [c, 0, a], rtol=1e-12, atol=1e-12)


def _quat_matrix_scipy(q):
    from scipy.spatial.transform import Rotation
    w, x, y, z = q
    return Rotation.from_quat([x, y, z, w]).as_matrix()


def test_projection_vs_numerical_jacobian(orc):
    """Sigma2 = J Sigma J^T + 0.3 I with J the numerical Jacobian of the pinhole
    map and Sigma from a library rotation; mean2d / depth from the pinhole map."""
    c = synth.config("c2", n=300, W=320, H=240)
    sc, cam = c["scene"], c["camera"]
    kp = orc.keypath(sc, cam)
    pr = orc.project(sc, cam, kp["tiles"])
    V = cam.view.astype(np.float64).reshape(3, 4)

    def pin(p):
        t = V[:, :3] @ p + V[:, 3]
        return np.array([cam.fx * t[0] / t[2] + cam.cx, cam.fy * t[1] / t[2] + cam.cy])

    lim = 1.3 * 0.5 * cam.W / cam.fx
    checked = 0
    for i in np.nonzero(kp["tiles"] > 0)[0][:100]:
        p = sc.means[i].astype(np.float64)
        t = V[:, :3] @ p + V[:, 3]
        if abs(t[0] / t[2]) > lim * 0.99 or abs(t[1] / t[2]) > 1.3 * 0.5 * cam.H / cam.fy * 0.99:
            continue
        J = np.zeros((2, 3))
        for k in range(3):
            e = np.zeros(3)
            e[k] = 1e-6
            J[:, k] = (pin(p + e) - pin(p - e)) / 2e-6
        R = _quat_matrix_scipy(sc.quats[i].astype(np.float64) / np.linalg.norm(sc.quats[i]))
        S = np.diag(np.exp(2 * sc.log_scales[i].astype(np.float64)))
        Sig2 = J @ R @ S @ R.T @ J.T + 0.3 * np.eye(2)
        np.testing.assert_allclose(pr["cov2d"][i], [Sig2[0, 0], Sig2[0, 1], Sig2[1, 1]], rtol=1e-6,
                                   atol=1e-6 * Sig2[0, 0])
        np.testing.assert_allclose(pr["mean2d"][i], pin(p), rtol=1e-12)
        assert abs(pr["depth"][i] - t[2]) < 1e-12
        checked += 1
    assert checked > 50


def test_keypath_fp32_agrees_with_fp64(orc):
    c = synth.config("c2", n=2000, W=320, H=240)
    sc, cam = c["scene"], c["camera"]
    kp = orc.keypath(sc, cam)
    pr = orc.project(sc, cam, kp["tiles"])
    v = kp["tiles"] > 0
    assert v.sum() > 500
    np.testing.assert_allclose(kp["mean2d"][v], pr["mean2d"][v], rtol=1e-5, atol=1e-3)
    np.testing.assert_allclose(kp["depth"][v], pr["depth"][v], rtol=1e-6)
    np.testing.assert_allclose(kp["cov2d"][v], pr["cov2d"][v], rtol=1e-4, atol=1e-4 * np.abs(pr["cov2d"][v]).max())


# --------------------------------------------------------------------------- compositing closed forms
def _pixel_center_mean(cam, px, py, z):
    return [(px - cam.cx) * z / cam.fx, (py - cam.cy) * z / cam.fy, z]


def test_two_gaussian_compositing(orc):
    cam = ident_camera(bg=(0.2, 0.3, 0.4))
    o1, o2 = 0.6, 0.7
    c1, c2 = np.array([0.9, 0.1, 0.2]), np.array([0.1, 0.8, 0.3])
    ls = [[math.log(0.02)] * 3] * 2
    for swap in (False, True):
        z1, z2 = (3.0, 4.0) if not swap else (4.0, 3.0)
        sc = tiny_scene([_pixel_center_mean(cam, 16, 16, z1), _pixel_center_mean(cam, 16, 16, z2)], ls,
                        opacity=[o1, o2], rgb=[c1, c2], feat=[[1] * 8, [3] * 8], unc=[0.25, 0.75])
        out = orc.forward(sc, cam)
        img = out["img"]
        if not swap:
            (fa, oa), (fb, ob) = (c1, o1), (c2, o2)
            ua, ub, va, vb = 1.0, 3.0, 0.25, 0.75
        else:
            (fa, oa), (fb, ob) = (c2, o2), (c1, o1)
            ua, ub, va, vb = 3.0, 1.0, 0.75, 0.25
        expect = fa * oa + fb * ob * (1 - oa) + cam.bg * (1 - oa) * (1 - ob)
        np.testing.assert_allclose(img["rgb"][:, 16, 16], expect, rtol=1e-6)
        np.testing.assert_allclose(img["feat"][:, 16, 16], ua * oa + ub * ob * (1 - oa), rtol=1e-6)
        np.testing.assert_allclose(img["unc"][16, 16], va * oa + vb * ob * (1 - oa), rtol=1e-6)
        np.testing.assert_allclose(img["T"][16, 16], (1 - oa) * (1 - ob), rtol=1e-6)
        assert img["n_contrib"][16, 16] == 2
        keys = out["keys"]
        # the nearer Gaussian comes first in its tile
        t = (16 // 16) * cam.tiles_x + 16 // 16
        s, e = out["ranges"][t]
        first = out["vals"][s]
        assert first == (0 if not swap else 1)


def test_partition_of_unity(orc):
    """Sum_i alpha_i T_i + T_final = 1: equal colours and bg = that colour render it exactly;
    equal features v render v (1 - T_final)."""
    c = synth.config("c1", n=500, W=64, H=64)
    sc = c["scene"]
    cam = c["camera"]
    col = np.array([0.3, 0.6, 0.9], np.float32)
    cam.bg = col.copy()
    sc.sh[:] = 0
    sc.sh[:, 0, :] = (col - 0.5) / Y00
    sc.feat[:] = 2.5
    sc.unc[:] = 0.4
    out = orc.forward(sc, cam)
    img = out["img"]
    for ch in range(3):
        np.testing.assert_allclose(img["rgb"][ch], col[ch], rtol=1e-6)
    np.testing.assert_allclose(img["feat"], np.broadcast_to(2.5 * (1 - img["T"]), img["feat"].shape),
                               rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(img["unc"], float(np.float32(0.4)) * (1 - img["T"]), rtol=1e-9, atol=1e-12)
    assert img["T"].min() >= 1e-4 and img["T"].max() <= 1.0


def test_termination_alpha_08(orc):
    """Identical alpha = 0.8 Gaussians on one pixel: T = 0.2^k; the sixth would
    give 6.4e-5 < 1e-4, so five are blended and T_final = 3.2e-4."""
    cam = ident_camera()
    n = 8
    sc = tiny_scene([_pixel_center_mean(cam, 16, 16, 2.0 + 0.1 * k) for k in range(n)],
                    [[math.log(0.02)] * 3] * n, opacity=[0.8] * n)
    img = orc.forward(sc, cam)["img"]
    assert img["n_contrib"][16, 16] == 5
    np.testing.assert_allclose(img["T"][16, 16], 0.2 ** 5, rtol=1e-6)  # FP32-stored opacity


# --------------------------------------------------------------------------- binning
def test_tiled_render_equals_brute_force(orc):
    c = synth.config("c1")
    sc, cam = c["scene"], c["camera"]
    out = orc.forward(sc, cam)
    tl = [(tx, ty) for ty in range(cam.tiles_y) for tx in range(cam.tiles_x)]
    vals_b, ranges_b = orc.lists_for_tiles(cam, out["kp"], tl)
    img_b = orc.render(cam, sc, out["proj"], vals_b, ranges_b)
    for k in ("rgb", "feat", "unc", "T", "n_contrib"):
        assert np.array_equal(out["img"][k], img_b[k]), k


def test_binning_invariants(orc):
    c = synth.config("c2", n=3000, W=160, H=120)
    sc, cam = c["scene"], c["camera"]
    kp = orc.keypath(sc, cam)
    keys, vals, ranges = orc.bin(cam, kp)
    assert np.all(keys[1:] >= keys[:-1])
    # multiset of (tile, id) equals the enumeration of every rectangle row's span
    want = []
    for i in np.nonzero(kp["tiles"] > 0)[0]:
        x0, y0, x1, y1 = kp["rect"][i]
        for ty in range(y0, y1):
            xl, xr = orc.row_span(kp, i, ty)
            assert x0 <= xl <= xr <= x1
            want.extend((ty * cam.tiles_x + tx, i) for tx in range(xl, xr))
    got = sorted(zip((keys >> np.uint64(32)).astype(np.int64).tolist(), vals.tolist()))
    assert got == sorted(want)
    # without the ellipse: the whole rectangles
    keys_r, vals_r, _ = orc.bin(cam, kp, ellipse=False)
    assert len(keys_r) == kp["tiles"].sum() > len(keys)
    assert orc.bin_count(kp) == len(keys) and orc.bin_count(kp, ellipse=False) == len(keys_r)
    # low word is the depth's float bits
    assert np.array_equal((keys & np.uint64(0xFFFFFFFF)).astype(np.uint32), kp["depth"].view(np.uint32)[vals])
    # ranges partition the sorted list by tile id
    tid = (keys >> np.uint64(32)).astype(np.int64)
    for t in range(cam.tiles_x * cam.tiles_y):
        s, e = ranges[t]
        if s == e:
            assert not np.any(tid == t)
        else:
            assert np.all(tid[s:e] == t) and (s == 0 or tid[s - 1] != t) and (e == len(tid) or tid[e] != t)
    # ties (equal depth) keep the lower index first
    for t in range(cam.tiles_x * cam.tiles_y):
        s, e = ranges[t]
        k = keys[s:e]
        v = vals[s:e]
        same = k[1:] == k[:-1]
        assert np.all(v[1:][same] > v[:-1][same])


# --------------------------------------------------------------------------- tile ellipse
def test_ln_up_bounds_ln(orc):
    xs = np.concatenate([np.geomspace(1e-3, 300.0, 20001), 2.0 ** np.arange(-9, 9),
                         np.nextafter(2.0 ** np.arange(-9, 9), 0)]).astype(np.float32)
    got = np.array([orc.ln_up_f32(float(x)) for x in xs], np.float64)
    ref = np.log(xs.astype(np.float64))
    assert np.all(got >= ref - 2e-6)                 # an upper bound up to FP32 rounding
    assert np.max(got - ref) < 0.0141                # and within 1/sqrt(2) - ln 2
    assert abs(orc.ln_up_f32(1.0)) == 0.0


def _aniso_scene(n, seed):
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-1.2, 1.2, n), rng.uniform(-0.9, 0.9, n), rng.uniform(2.0, 4.0, n)], 1)
    ls = np.stack([rng.normal(-2.2, 0.6, n), rng.normal(-3.5, 0.6, n), rng.normal(-3.0, 0.5, n)], 1)
    q = rng.standard_normal((n, 4))
    o = np.concatenate([rng.uniform(0.003, 0.999, n - 8), [1 / 255 * 0.9, 1 / 255 * 1.01, 0.999, 0.9995,
                                                          0.01, 0.02, 0.5, 0.99]])
    sc = tiny_scene(means, ls, quats=q / np.linalg.norm(q, axis=1, keepdims=True), opacity=o)
    return sc


def test_tile_ellipse_complete_and_tight(orc):
    """Every tile with a pixel at alpha >= 1/255 (FP64) is binned; every binned
    tile's box, widened by half a pixel, reaches q <= 2 ln(255 o) + 0.2 (0.25 px grid)."""
    W, H = 160, 128
    cam = ident_camera(W, H, f=110.0)
    sc = _aniso_scene(400, 3)
    kp = orc.keypath(sc, cam)
    pr = orc.project(sc, cam, kp["tiles"])
    keys, vals, _ = orc.bin(cam, kp)
    binned = set(zip((keys >> np.uint64(32)).astype(np.int64).tolist(), vals.tolist()))
    TX = cam.tiles_x
    n_rect = n_kept = 0
    gx = np.arange(-0.5, 16.0, 0.25)
    for i in np.nonzero(kp["tiles"] > 0)[0]:
        A, B, Cc = pr["conic"][i]
        mx, my = pr["mean2d"][i]
        o = pr["opacity"][i]
        lim = 2 * math.log(255 * o)
        x0, y0, x1, y1 = kp["rect"][i]
        for ty in range(y0, y1):
            for tx in range(x0, x1):
                n_rect += 1
                kept = (ty * TX + tx, i) in binned
                n_kept += kept
                px, py = np.meshgrid(np.arange(16.0) + 16 * tx, np.arange(16.0) + 16 * ty)
                dx, dy = mx - px, my - py
                alpha = o * np.exp(-0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy)
                if alpha.max() >= 1 / 255:
                    assert kept, (i, tx, ty, alpha.max())
                if kept:
                    qx, qy = np.meshgrid(gx + 16 * tx, gx + 16 * ty)
                    ex, ey = mx - qx, my - qy
                    qmin = (A * ex * ex + 2 * B * ex * ey + Cc * ey * ey).min()
                    assert qmin <= lim + 0.2, (i, tx, ty, qmin, lim)
    assert n_kept < 0.8 * n_rect


def test_ellipse_binning_renders_like_rectangles(orc):
    """Left-out tiles hold no pixel with alpha >= 1/255, so images, transmittance
    and all gradients equal those of whole-rectangle binning exactly (FP64)."""
    W, H = 160, 128
    cam = ident_camera(W, H, f=110.0, bg=(0.1, 0.2, 0.3))
    sc = _aniso_scene(400, 4)
    kp = orc.keypath(sc, cam)
    pr = orc.project(sc, cam, kp["tiles"])
    _, ve, re_ = orc.bin(cam, kp)
    _, vr, rr = orc.bin(cam, kp, ellipse=False)
    assert len(ve) < len(vr)
    ie, ir = orc.render(cam, sc, pr, ve, re_), orc.render(cam, sc, pr, vr, rr)
    for k in ("rgb", "feat", "unc", "T", "flip"):
        assert np.array_equal(ie[k], ir[k]), k
    assert np.all(ie["n_contrib"] <= ir["n_contrib"])
    rng = np.random.default_rng(1)
    dr, df, du = rng.standard_normal((3, H, W)), rng.standard_normal((8, H, W)), rng.standard_normal((H, W))
    ge = orc.render_bwd(cam, sc, pr, ve, re_, dr, df, du)
    gr = orc.render_bwd(cam, sc, pr, vr, rr, dr, df, du)
    for k in ge:
        assert np.array_equal(ge[k], gr[k]), k


# --------------------------------------------------------------------------- backward: finite differences
def test_render_bwd_matches_fd(orc):
    c = synth.config("c1", n=300, W=64, H=64)
    sc, cam = c["scene"], c["camera"]
    cam.bg = np.array([0.1, 0.2, 0.3], np.float32)
    out = orc.forward(sc, cam)
    proj, vals, ranges = out["proj"], out["vals"], out["ranges"]
    rng = np.random.default_rng(5)
    dr, df, du = rng.standard_normal((3, 64, 64)), rng.standard_normal((8, 64, 64)), rng.standard_normal((64, 64))

    def loss(pr, scn):
        im = orc.render(cam, scn, pr, vals, ranges)
        return (im["rgb"] * dr).sum() + (im["feat"] * df).sum() + (im["unc"] * du).sum()

    g = orc.render_bwd(cam, sc, proj, vals, ranges, dr, df, du)
    vis = np.nonzero(out["kp"]["tiles"] > 0)[0]
    pick = rng.choice(vis, 12, replace=False)
    for i in pick:
        for key, n in (("mean2d", 2), ("conic", 3), ("opacity", 1), ("rgb", 3)):
            for k in range(n):
                h = 1e-6 * max(1.0, abs(proj[key].reshape(len(proj[key]), -1)[i, k]))
                pp = {kk: vv.copy() for kk, vv in proj.items()}
                pm = {kk: vv.copy() for kk, vv in proj.items()}
                pp[key].reshape(len(pp[key]), -1)[i, k] += h
                pm[key].reshape(len(pm[key]), -1)[i, k] -= h
                fd = (loss(pp, sc) - loss(pm, sc)) / (2 * h)
                an = g[key].reshape(len(g[key]), -1)[i, k]
                assert abs(fd - an) <= 1e-5 * max(1.0, abs(fd)), (key, i, k, fd, an)
        # features and uncertainty enter linearly: the derivative is exact blending weight
        for k in range(8):
            sp = synth.Scene(**{**sc.__dict__, "feat": sc.feat.copy()})
            sp.feat[i, k] += 1.0
            fd = loss(proj, sp) - loss(proj, sc)
            assert abs(fd - g["feat"][i, k]) < 1e-6 * max(1.0, abs(fd))


def test_project_bwd_matches_fd(orc):
    c = synth.config("c2", n=400, W=320, H=240)
    sc, cam = c["scene"], c["camera"]
    kp = orc.keypath(sc, cam)
    tiles = kp["tiles"]
    rng = np.random.default_rng(6)
    N = sc.N
    w = dict(mean2d=rng.standard_normal((N, 2)), conic=rng.standard_normal((N, 3)) * 100,
             opacity=rng.standard_normal(N), rgb=rng.standard_normal((N, 3)))

    def L(s):
        p = orc.project(s, cam, tiles)
        return sum((p[k] * w[k]).sum() for k in w), p

    base, pr = L(sc)
    g = orc.project_bwd(sc, cam, tiles, w["mean2d"], w["conic"], w["opacity"], w["rgb"])
    vis = np.nonzero(tiles > 0)[0]
    pick = rng.choice(vis, 10, replace=False)
    for i in pick:
        for key in ("means", "log_scales", "quats", "opacity_raw", "sh"):
            arr = getattr(sc, key).astype(np.float64)
            flat_n = arr.reshape(N, -1).shape[1]
            for k in range(flat_n):
                h = 1e-6
                sp = synth.Scene(**{**sc.__dict__, key: arr.copy()})
                sm = synth.Scene(**{**sc.__dict__, key: arr.copy()})
                getattr(sp, key).reshape(N, -1)[i, k] += h
                getattr(sm, key).reshape(N, -1)[i, k] -= h
                fd = (L(sp)[0] - L(sm)[0]) / (2 * h)
                an = g[key].reshape(N, -1)[i, k]
                assert abs(fd - an) <= 2e-6 * max(1.0, abs(fd)), (key, i, k, fd, an)


# --------------------------------------------------------------------------- decoder
def test_decoder_matches_library(orc):
    from scipy.special import logsumexp, softmax
    dec = synth.decoder_init(7, 32)
    rng = np.random.default_rng(7)
    f = rng.standard_normal((8, 200))
    z = orc.decoder_fwd(f, dec)
    W1, b1, W2, b2, W3, b3 = [a.astype(np.float64) for a in (dec.W1, dec.b1, dec.W2, dec.b2, dec.W3, dec.b3)]
    h1 = np.maximum(W1 @ f + b1[:, None], 0)
    h2 = np.maximum(W2 @ h1 + b2[:, None], 0)
    np.testing.assert_allclose(z, W3 @ h2 + b3[:, None], rtol=1e-12, atol=1e-12)
    prob, am = orc.softmax_argmax(z)
    np.testing.assert_allclose(prob, softmax(z, axis=0), rtol=1e-12)
    assert np.array_equal(am, np.argmax(z, axis=0))
    tgt = rng.integers(0, 32, 200)
    u = rng.uniform(0, 1, 200)
    out = orc.decoder_loss(f, u, tgt, dec, 1.0, 1.0)
    ce = logsumexp(z, axis=0) - z[tgt, np.arange(200)]
    np.testing.assert_allclose(out["loss"], [(ce * (1 - u)).mean(), u.mean()], rtol=1e-12)


def test_decoder_argmax_ties_lowest():
    # ties -> lowest index (closed form on a hand-made logit column)
    import oracle
    z = np.array([[1.0], [3.0], [3.0], [2.0]])
    _, am = oracle.softmax_argmax(z)
    assert am[0] == 1


def test_decoder_loss_fd(orc):
    dec = synth.decoder_init(8, 16)
    rng = np.random.default_rng(8)
    P = 50
    f = rng.standard_normal((8, P))
    u = rng.uniform(0, 1, P)
    tgt = rng.integers(0, 16, P)
    lce, lu = 1.0, 0.7

    def Ls(ff, uu, d):
        o = orc.decoder_loss(ff, uu, tgt, d, lce, lu)
        return lce * o["loss"][0] + lu * o["loss"][1]

    g = orc.decoder_loss(f, u, tgt, dec, lce, lu)
    h = 1e-6
    for p in range(0, P, 7):
        for k in range(8):
            fp, fm = f.copy(), f.copy()
            fp[k, p] += h
            fm[k, p] -= h
            fd = (Ls(fp, u, dec) - Ls(fm, u, dec)) / (2 * h)
            assert abs(fd - g["d_feat"][k, p]) < 1e-7 * max(1, abs(fd))
        up, um = u.copy(), u.copy()
        up[p] += h
        um[p] -= h
        fd = (Ls(f, up, dec) - Ls(f, um, dec)) / (2 * h)
        assert abs(fd - g["d_unc"][p]) < 1e-7 * max(1, abs(fd))
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        arr = getattr(dec, name)
        flat = arr.reshape(-1)
        for idx in rng.choice(flat.size, 5, replace=False):
            d64 = synth.Decoder(**{k: v.astype(np.float64) for k, v in dec.__dict__.items()})
            dp = synth.Decoder(**{k: v.copy() for k, v in d64.__dict__.items()})
            dm = synth.Decoder(**{k: v.copy() for k, v in d64.__dict__.items()})
            getattr(dp, name).reshape(-1)[idx] += h
            getattr(dm, name).reshape(-1)[idx] -= h
            fd = (Ls(f, u, dp) - Ls(f, u, dm)) / (2 * h)
            an = g["d" + name].reshape(-1)[idx]
            assert abs(fd - an) < 1e-7 * max(1, abs(fd)), (name, idx, fd, an)


# --------------------------------------------------------------------------- query
def test_relevancy_closed_form(orc):
    rng = np.random.default_rng(9)
    d_clip, d = 16, 24
    q = synth.unit_rows(rng, 2, d_clip)
    negs = synth.unit_rows(rng, 3, d_clip)
    cb = synth.unit_rows(rng, 5, d)
    # entry 2's CLIP part is parallel to text 0
    cb[2, :d_clip] = 0.7 * q[0]
    qin = synth.QueryInputs(cb, q, negs, d_clip)
    prob = np.zeros((5, 3))
    prob[2, 0] = 1.0                           # one-hot: F = S_2, phi = q_0
    prob[:, 1] = 0.2                           # uniform: F = mean of rows
    prob[0, 2] = 1.0
    rel = orc.query(prob, qin)
    q0 = q[0].astype(np.float64)
    s2 = cb[2, :d_clip].astype(np.float64)       # one-hot: F = S_2, parallel to q_0 up to FP32 rounding
    phi0 = s2 / np.linalg.norm(s2)
    sq = float(phi0 @ q0)
    want = min(math.exp(sq) / (math.exp(sq) + math.exp(float(phi0 @ n))) for n in negs.astype(np.float64))
    assert abs(rel[0, 0] - want) < 1e-12
    assert abs(want - min(math.e / (math.e + math.exp(float(q0 @ n))) for n in negs)) < 1e-6
    F = cb.astype(np.float64).mean(0)[:d_clip]
    phi = F / np.linalg.norm(F)
    for j in range(2):
        w = min(1 / (1 + math.exp(float(phi @ n) - float(phi @ q[j]))) for n in negs)
        assert abs(rel[j, 1] - w) < 1e-12
    # a text equal to a negative has relevancy <= 1/2
    qin2 = synth.QueryInputs(cb, negs[:1].copy(), negs, d_clip)
    rel2 = orc.query(prob, qin2)
    assert np.all(rel2 <= 0.5 + 1e-15)


# --------------------------------------------------------------------------- training
def test_adam_first_step_and_torch(orc):
    import torch
    rng = np.random.default_rng(10)
    g = rng.standard_normal(100)
    p = rng.standard_normal(100)
    m = np.zeros(100)
    v = np.zeros(100)
    p1 = p.copy()
    orc.adam(p1, g, m, v, 1)
    np.testing.assert_allclose(p1, p - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
    # five steps against torch.optim.Adam (CPU, float64)
    tp = torch.tensor(p, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    p2, m2, v2 = p.copy(), np.zeros(100), np.zeros(100)
    for step in range(1, 6):
        gs = rng.standard_normal(100)
        tp.grad = torch.tensor(gs)
        opt.step()
        orc.adam(p2, gs, m2, v2, step)
    np.testing.assert_allclose(p2, tp.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_l1(orc):
    img = np.array([0.5, 0.25, 0.875, 0.375])
    tgt = np.array([0.25, 0.25, 1.0, 0.0], np.float32)
    loss, g = orc.l1(img, tgt)
    assert loss == (0.25 + 0 + 0.125 + 0.375) / 4
    np.testing.assert_array_equal(g, [0.25, 0, -0.25, 0.25])


# ---------------------------------------------------------------------------
# Quantisation of language features (Sec. 3.3, supp. "Load Balancing Loss")

def _bf16_torch_bits(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(torch.bfloat16).view(torch.int16).numpy() \
        .view(np.uint16)


def test_bf16_rounding_matches_torch(orc):
    rng = np.random.default_rng(30)
    x = (rng.standard_normal(20000) * 10.0 ** rng.integers(-6, 6, 20000)).astype(np.float32)
    # exact ties between two BF16 neighbours (round half to even; finite values) and signed zeros
    ties = (rng.integers(0, 0x7F7F, 2000).astype(np.uint32) << 16) | np.uint32(0x8000)
    x = np.concatenate([x, ties.view(np.float32), -ties.view(np.float32), np.array([0.0, -0.0, 1.0, -3.5], np.float32)])
    assert x.dtype == np.float32 and np.all(np.isfinite(x))
    assert np.array_equal(orc.bf16_bits(x), _bf16_torch_bits(x))


def _split_cos(A, B, d_clip):
    from scipy.spatial.distance import cdist
    return 1.0 - cdist(A[:, :d_clip], B[:, :d_clip], "cosine"), 1.0 - cdist(A[:, d_clip:], B[:, d_clip:], "cosine")


def _bf16_value(bits):
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def test_quant_distance_vs_library_cosine(orc):
    rng = np.random.default_rng(31)
    K, N, d, dc = 300, 32, 896, 512
    S = rng.standard_normal((N, d)).astype(np.float32)
    F = orc.bf16_bits(rng.standard_normal((K, d)))
    o = orc.quantize(F, S, want_D=True)
    cc, cd = _split_cos(_bf16_value(F), _bf16_value(orc.bf16_bits(S)), dc)
    D = cc + 0.5 * cd
    assert np.abs(o["D"] - D).max() < 1e-12
    assert np.array_equal(o["m"], np.argmax(D, axis=1))
    best = D[np.arange(K), o["m"]]
    assert abs(o["loss"][1] - np.mean(1.5 - best)) < 1e-12            # L_cos = 1 + lambda_D - D(F, f_m)


def test_quant_feature_equal_to_code(orc):
    """F_i = f_j exactly: both cosines are 1, D = 1 + lambda_D is the maximum, m_i = j, L_cos = 0."""
    rng = np.random.default_rng(32)
    N, d = 64, 896
    S = rng.standard_normal((N, d)).astype(np.float32)
    pick = rng.integers(0, N, 500)
    F = orc.bf16_bits(S)[pick]
    o = orc.quantize(F, S, want_D=True)
    assert np.array_equal(o["m"], pick)
    assert np.abs(o["D"][np.arange(500), pick] - 1.5).max() < 1e-12
    assert abs(o["loss"][1]) < 1e-12


def test_quant_load_balance_closed_form(orc):
    """Orthonormal codes e_j in both parts and features equal to codes: D = (1 + lambda_D) delta_ij,
    each softmax row puts a = e^1.5/(e^1.5 + N - 1) on its own code and b = 1/(e^1.5 + N - 1)
    elsewhere, so with c_j features on code j: r_j = c_j/K, p_j = (c_j a + (K - c_j) b)/K and
    L_lb = sum_j r_j p_j; a balanced split gives L_lb = 1/N."""
    N, d, dc = 16, 896, 512
    S = np.zeros((N, d), np.float32)
    for j in range(N):
        S[j, j] = 1.0
        S[j, dc + j] = 1.0
    e = np.exp(1.5)
    a, b = e / (e + N - 1), 1.0 / (e + N - 1)
    for counts in (np.full(N, 7), np.arange(1, N + 1)):
        pick = np.repeat(np.arange(N), counts)
        K = len(pick)
        o = orc.quantize(orc.bf16_bits(S[pick]), S)
        r = counts / K
        p = (counts * a + (K - counts) * b) / K
        assert np.allclose(o["r"], r, rtol=0, atol=1e-15)
        assert np.allclose(o["p"], p, rtol=0, atol=1e-14)
        assert abs(o["loss"][2] - np.sum(r * p)) < 1e-14
        assert abs(o["loss"][0] - (o["loss"][1] + 0.5 * o["loss"][2])) < 1e-14   # L_q, lambda_cos = 1
    assert abs(np.sum(np.full(N, 1.0 / N) ** 2) - 1.0 / N) < 1e-15


def test_quant_codebook_gradient_fd(orc):
    """dL_q/dS against central differences of L_q (argmax winners, and with them r, unchanged)."""
    rng = np.random.default_rng(33)
    K, N, d, dc = 40, 8, 48, 32
    S = rng.standard_normal((N, d))
    F = orc.bf16_bits(S[rng.integers(0, N, K)] + 0.7 * rng.standard_normal((K, d)))
    o = orc.quantize(F, S, d_clip=dc, round_codebook=False, want_grad=True)
    G = o["grad_S"]
    h = 1e-6
    for j, e in [(int(rng.integers(N)), int(rng.integers(d))) for _ in range(40)]:
        Sp, Sm = S.copy(), S.copy()
        Sp[j, e] += h
        Sm[j, e] -= h
        op = orc.quantize(F, Sp, d_clip=dc, round_codebook=False)
        om = orc.quantize(F, Sm, d_clip=dc, round_codebook=False)
        assert np.array_equal(op["m"], o["m"]) and np.array_equal(om["m"], o["m"])
        fd = (op["loss"][0] - om["loss"][0]) / (2 * h)
        assert abs(fd - G[j, e]) <= 1e-6 * max(1.0, np.abs(G).max()), (j, e, fd, G[j, e])


# ---------------------------------------------------------------------------
# Adaptive spatial smoothing (Sec. 3.4, Eqs. eq:lem_fmlp, eq:lem_loss_mlp; supp. Tab. pemlp)

def _smooth_case(n=6, seed=40):
    from paper_2311_18482_gb300 import synth
    rng = np.random.default_rng(seed)
    mlp = synth.smooth_mlp_init(seed)
    P = {k: getattr(mlp, k).astype(np.float64) for k in ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")}
    means = rng.uniform(-1, 1, (n, 3))
    feat = rng.standard_normal((n, 8))
    unc = rng.uniform(0, 0.3, n)          # some below w_s = 0.1, some above
    return P, means, feat, unc


def _mlp_np(P, x):
    h = np.maximum(x @ P["W1"].T + P["b1"], 0)
    h = np.maximum(h @ P["W2"].T + P["b2"], 0)
    h = np.maximum(h @ P["W3"].T + P["b3"], 0)
    return h @ P["W4"].T + P["b4"]


def test_smooth_forward_vs_numpy(orc):
    P, means, feat, unc = _smooth_case(50)
    o = orc.smooth(means, feat, unc, P, w_s=0.1, lam=0.7)
    s = _mlp_np(P, means)
    assert np.abs(o["s_mlp"] - s).max() < 1e-12
    nrm = np.linalg.norm(s - feat, axis=1)
    assert abs(o["loss"] - 0.7 * np.mean((1 + np.maximum(unc, 0.1)) * nrm)) < 1e-12


def test_smooth_gradients_fd(orc):
    """The stop-gradients split L_smo into T1 = |s_MLP(W) - s_G*| (MLP parameters) and
    T2 = max(u*, w_s) |s_MLP* - s_G| (semantic features); each gradient is checked by
    central differences of its own term."""
    P, means, feat, unc = _smooth_case(6)
    lam, ws = 0.9, 0.1
    o = orc.smooth(means, feat, unc, P, w_s=ws, lam=lam)
    wgt = np.maximum(unc, ws)

    def t1(Q):
        return lam * np.mean(np.linalg.norm(_mlp_np(Q, means) - feat, axis=1))

    def t2(f):
        return lam * np.mean(wgt * np.linalg.norm(o["s_mlp"] - f, axis=1))

    assert abs(o["loss"] - (t1(P) + t2(feat))) < 1e-12
    rng = np.random.default_rng(41)
    h = 1e-6
    for k in ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4"):
        for _ in range(6):
            idx = tuple(int(rng.integers(s)) for s in P[k].shape)
            Qp = {kk: v.copy() for kk, v in P.items()}
            Qm = {kk: v.copy() for kk, v in P.items()}
            Qp[k][idx] += h
            Qm[k][idx] -= h
            fd = (t1(Qp) - t1(Qm)) / (2 * h)
            assert abs(fd - o["d" + k][idx]) <= 1e-6 * max(1.0, np.abs(o["d" + k]).max()), (k, idx)
    for _ in range(10):
        i, c = int(rng.integers(6)), int(rng.integers(8))
        fp, fm = feat.copy(), feat.copy()
        fp[i, c] += h
        fm[i, c] -= h
        fd = (t2(fp) - t2(fm)) / (2 * h)
        assert abs(fd - o["d_feat"][i, c]) <= 1e-7


def test_smooth_closed_forms(orc):
    """W4 = 0: s_MLP = b4 for every Gaussian.  With s_G = b4 the loss and all gradients are 0
    (zero-difference reading); with s_G = b4 - e_c the difference is a unit vector, so
    L = lam mean(1 + max(u, w_s)), dL/db4 = lam e_c and dL/ds_G = -lam max(u, w_s) e_c / n."""
    P, means, feat, unc = _smooth_case(7)
    P["W4"][:] = 0.0
    f0 = np.tile(P["b4"], (7, 1))
    o = orc.smooth(means, f0, unc, P, w_s=0.1, lam=1.0)
    assert o["loss"] == 0.0 and not np.any(o["d_feat"]) and not np.any(o["db4"]) and not np.any(o["dW1"])
    f1 = f0.copy()
    f1[:, 3] -= 1.0
    o = orc.smooth(means, f1, unc, P, w_s=0.1, lam=2.0)
    wgt = np.maximum(unc, 0.1)
    assert abs(o["loss"] - 2.0 * np.mean(1 + wgt)) < 1e-12
    e = np.zeros(8)
    e[3] = 1.0
    assert np.abs(o["db4"] - 2.0 * e).max() < 1e-12
    assert np.abs(o["d_feat"] - (-2.0 / 7) * wgt[:, None] * e).max() < 1e-12


def test_feature_map_pins(orc):
    """F = M_infer S (supp. "Inference"): a one-hot distribution returns its code exactly; a
    general one equals the library matrix product."""
    rng = np.random.default_rng(50)
    N, P, d = 32, 40, 896
    S = rng.standard_normal((N, d)).astype(np.float32)
    onehot = np.zeros((N, P))
    m = rng.integers(0, N, P)
    onehot[m, np.arange(P)] = 1.0
    assert np.array_equal(orc.feature_map(onehot, S), S[m].astype(np.float64))
    prob = rng.dirichlet(np.ones(N), P).T
    assert np.abs(orc.feature_map(prob, S) - prob.T @ S.astype(np.float64)).max() < 1e-12


# ---------------------------------------------------------------------------
# RGB loss with D-SSIM (3DGS's loss, kept by Sec. 4)

def _window11():
    g = np.exp(-np.arange(-5, 6) ** 2 / (2 * 1.5 ** 2))
    return np.outer(g, g) / g.sum() ** 2


def test_ssim_map_vs_library_filter(orc):
    """The SSIM map from scipy's correlate with the same window and zero padding."""
    from scipy.ndimage import correlate
    rng = np.random.default_rng(60)
    x, y = rng.uniform(0, 1, (3, 23, 31)), rng.uniform(0, 1, (3, 23, 31))
    o = orc.rgb_loss(x, y, want_map=True)
    w = _window11()
    f = lambda a: correlate(a, w, mode="constant", cval=0.0)
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    for c in range(3):
        mx, my = f(x[c]), f(y[c])
        vx, vy, cxy = f(x[c] ** 2) - mx ** 2, f(y[c] ** 2) - my ** 2, f(x[c] * y[c]) - mx * my
        S = (2 * mx * my + C1) * (2 * cxy + C2) / ((mx ** 2 + my ** 2 + C1) * (vx + vy + C2))
        assert np.abs(o["smap"][c] - S).max() < 1e-12
    assert abs(o["loss"][2] - o["smap"].mean()) < 1e-14
    assert abs(o["loss"][1] - np.abs(x - y).mean()) < 1e-14
    assert abs(o["loss"][0] - (0.8 * o["loss"][1] + 0.2 * (1 - o["loss"][2]))) < 1e-14


def test_ssim_closed_forms(orc):
    """SSIM(x, x) = 1 everywhere (L = 0, gradient 0); constant images a, b away from the border:
    S = (2ab + C1)/(a^2 + b^2 + C1)."""
    rng = np.random.default_rng(61)
    x = rng.uniform(0, 1, (3, 20, 24))
    o = orc.rgb_loss(x, x, want_map=True)
    assert np.abs(o["smap"] - 1).max() < 1e-12 and abs(o["loss"][0]) < 1e-12
    assert np.abs(o["grad"]).max() < 1e-12
    a, b = 0.3, 0.7
    o = orc.rgb_loss(np.full((3, 30, 30), a), np.full((3, 30, 30), b), want_map=True)
    C1 = 0.01 ** 2
    assert np.abs(o["smap"][:, 5:-5, 5:-5] - (2 * a * b + C1) / (a * a + b * b + C1)).max() < 1e-12


def test_ssim_gradient_fd(orc):
    rng = np.random.default_rng(62)
    x, y = rng.uniform(0, 1, (3, 14, 17)), rng.uniform(0, 1, (3, 14, 17))
    o = orc.rgb_loss(x, y, lam=0.2)
    h = 1e-6
    for _ in range(25):
        c, i, j = int(rng.integers(3)), int(rng.integers(14)), int(rng.integers(17))
        xp, xm = x.copy(), x.copy()
        xp[c, i, j] += h
        xm[c, i, j] -= h
        fd = (orc.rgb_loss(xp, y, want_grad=False)["loss"][0] - orc.rgb_loss(xm, y, want_grad=False)["loss"][0]) / (2 * h)
        assert abs(fd - o["grad"][c, i, j]) <= 1e-8 + 1e-6 * abs(fd), (c, i, j, fd, o["grad"][c, i, j])


# ---------------------------------------------------------------------------
# Adaptive density control (3DGS's clone / split / prune, kept by Sec. 4)

def test_densify_stats_hand_case(orc):
    """Two steps of the statistics on three Gaussians, worked by hand: 3-4-5 and
    6-8-10 triangles give exact FP32 norms; a Gaussian with radius 0 (outside
    the view) is neither accumulated nor counted.  Accumulating |g|^2, only one
    component, or counting radius-0 Gaussians each changes an entry."""
    acc = np.zeros(3, np.float32)
    cnt = np.zeros(3, np.int32)
    orc.densify_stats(np.array([[3, 4], [0.5, -1.25], [6, 8]], np.float32), np.array([2, 0, 1]), acc, cnt)
    assert acc.tolist() == [5.0, 0.0, 10.0] and cnt.tolist() == [1, 0, 1]
    orc.densify_stats(np.array([[-6, -8], [1, 1], [5, 12]], np.float32), np.array([1, 5, 0]), acc, cnt)
    assert acc.tolist() == [15.0, float(np.float32(np.sqrt(np.float32(2)))), 10.0]
    assert cnt.tolist() == [2, 1, 1]


def test_densify_stats_vs_hypot(orc):
    """Three steps on random gradients against numpy's hypot summed in FP64: the
    oracle's FP32 norm and sum stay within a few FP32 roundings of it."""
    rng = np.random.default_rng(83)
    n = 20000
    acc = np.zeros(n, np.float32)
    cnt = np.zeros(n, np.int32)
    ref = np.zeros(n)
    ref_cnt = np.zeros(n, np.int64)
    for _ in range(3):
        g = (rng.standard_normal((n, 2)) * 10.0 ** rng.uniform(-6, 0, (n, 1))).astype(np.float32)
        rad = rng.integers(0, 3, n).astype(np.int32)
        orc.densify_stats(g, rad, acc, cnt)
        vis = rad > 0
        ref[vis] += np.hypot(g[vis, 0].astype(np.float64), g[vis, 1].astype(np.float64))
        ref_cnt[vis] += 1
    assert np.array_equal(cnt, ref_cnt)
    err = np.abs(acc.astype(np.float64) - ref)
    assert np.all(err <= 4 * 2.0 ** -24 * ref + 1e-30), err.max()
    assert np.all((ref == 0) == (acc == 0))


def _densify_inputs(n, seed):
    rng = np.random.default_rng(seed)
    P = {"means": rng.uniform(-1, 1, (n, 3)).astype(np.float32),
         "log_scales": rng.normal(-3, 1, (n, 3)).astype(np.float32),
         "quats": rng.standard_normal((n, 4)).astype(np.float32),
         "opacity_raw": rng.normal(0, 3, n).astype(np.float32),
         "sh": rng.standard_normal((n, 16, 3)).astype(np.float32),
         "feat": rng.standard_normal((n, 8)).astype(np.float32),
         "unc": rng.uniform(0, 1, n).astype(np.float32)}
    acc = rng.uniform(0, 0.004, n).astype(np.float32)
    cnt = rng.integers(0, 10, n).astype(np.int32)
    return P, acc, cnt


def test_densify_plan_matches_definitions(orc):
    """The FP32 threshold forms take the same decisions as the definitions (sigmoid, mean gradient,
    exp of the largest log-scale) evaluated in FP64, away from the thresholds."""
    P, acc, cnt = _densify_inputs(4000, 70)
    noise = np.zeros((4000, 2, 3), np.float32)
    o = orc.densify(P, P, P, acc, cnt, noise, grad_thresh=0.0002, percent_dense=0.01, extent=4.0, min_opacity=0.005)
    op = 1 / (1 + np.exp(-P["opacity_raw"].astype(np.float64)))
    g = np.where(cnt > 0, acc / np.maximum(cnt, 1), 0.0)
    big = np.exp(P["log_scales"].astype(np.float64).max(1)) > 0.01 * 4.0
    want = np.where(op < 0.005, 0, np.where((cnt > 0) & (g >= 0.0002), np.where(big, 3, 2), 1))
    far = (np.abs(op - 0.005) > 1e-6) & (np.abs(g - 0.0002) > 1e-9) & \
          (np.abs(np.exp(P["log_scales"].astype(np.float64).max(1)) - 0.04) > 1e-7)
    assert np.array_equal(o["kind"][far], want[far])
    assert len(set(o["kind"].tolist())) == 4                    # every kind occurs
    assert o["n_out"] == int(np.sum(want == 1) + 2 * np.sum(want >= 2))


def test_densify_size_pruning_matches_definitions(orc):
    """With 3DGS's size pruning on (largest screen radius > 20 px, largest scale > 0.1 x extent),
    the decisions equal the definitions evaluated in FP64 away from the thresholds; a Gaussian
    too large is pruned even when its gradient asks for a clone or split, and turning either
    test off brings back the plain decisions."""
    n = 4000
    P, acc, cnt = _densify_inputs(n, 72)
    rng = np.random.default_rng(73)
    P["log_scales"] = rng.normal(-1.5, 1.0, (n, 3)).astype(np.float32)
    mr = rng.integers(0, 40, n).astype(np.int32)
    noise = np.zeros((n, 2, 3), np.float32)
    kw = dict(grad_thresh=0.0002, percent_dense=0.01, extent=4.0, min_opacity=0.005)
    o = orc.densify(P, P, P, acc, cnt, noise, max_radius=mr, max_screen_size=20.0, world_frac=0.1, **kw)
    op = 1 / (1 + np.exp(-P["opacity_raw"].astype(np.float64)))
    g = np.where(cnt > 0, acc / np.maximum(cnt, 1), 0.0)
    smax = np.exp(P["log_scales"].astype(np.float64).max(1))
    pruned = (op < 0.005) | (mr > 20) | (smax > 0.1 * 4.0)
    want = np.where(pruned, 0, np.where((cnt > 0) & (g >= 0.0002), np.where(smax > 0.01 * 4.0, 3, 2), 1))
    far = (np.abs(op - 0.005) > 1e-6) & (np.abs(g - 0.0002) > 1e-9) & (np.abs(smax - 0.04) > 1e-7) & \
          (np.abs(smax - 0.4) > 1e-6)
    assert np.array_equal(o["kind"][far], want[far])
    for why in ((mr > 20), (smax > 0.4)):                   # each size test prunes Gaussians on its own
        assert np.any(why & (op >= 0.005) & far)
    o_off = orc.densify(P, P, P, acc, cnt, noise, **kw)
    plain = np.where(op < 0.005, 0, np.where((cnt > 0) & (g >= 0.0002), np.where(smax > 0.04, 3, 2), 1))
    assert np.array_equal(o_off["kind"][far], plain[far])
    assert np.any(o["kind"] != o_off["kind"])


def test_densify_max_radius_statistic(orc):
    """The largest screen radius since the statistics were reset, over three steps by hand;
    a Gaussian outside the view (radius 0) keeps its value."""
    acc = np.zeros(3, np.float32)
    cnt = np.zeros(3, np.int32)
    mr = np.zeros(3, np.int32)
    g = np.ones((3, 2), np.float32)
    for r in ([3, 0, 25], [7, 0, 4], [5, 2, 0]):
        orc.densify_stats(g, np.array(r, np.int32), acc, cnt, mr)
    assert mr.tolist() == [7, 2, 25] and cnt.tolist() == [3, 1, 2]


def test_opacity_reset(orc):
    """3DGS's opacity reset: sigmoid(opacity_raw') = min(sigmoid(opacity_raw), 0.01) in FP64 up to the
    FP32 rounding of the threshold; values already below are left bit for bit; the opacity's Adam
    moments restart at zero."""
    rng = np.random.default_rng(74)
    raw = np.concatenate([rng.normal(0, 4, 5000), [-4.59512, -4.59511, -20.0, 30.0]]).astype(np.float32)
    m = rng.standard_normal(len(raw)).astype(np.float32)
    v = rng.uniform(0, 1, len(raw)).astype(np.float32)
    r2 = raw.copy()
    orc.opacity_reset(r2, m, v, 0.01)
    sig = lambda x: 1 / (1 + np.exp(-x.astype(np.float64)))
    assert np.all(np.abs(sig(r2) - np.minimum(sig(raw), 0.01)) <= 0.01 * 1e-6)
    low = sig(raw) < 0.01 * (1 - 1e-6)
    assert np.array_equal(r2[low].view(np.uint32), raw[low].view(np.uint32))
    assert np.all(r2[~low] == orc.opacity_logit(0.01))
    assert np.all(m == 0) and np.all(v == 0)


def test_densify_layout_and_children(orc):
    """Output order (kept, clones, split children), moments carried or zeroed, child means
    mu + R diag(s) n: with n = +-e_k the child sits at distance s_k along R's k-th column."""
    P, acc, cnt = _densify_inputs(5, 71)
    P["opacity_raw"][:] = [5, -9, 5, 5, 5]                      # Gaussian 1 is pruned
    P["log_scales"][:] = -4.0
    P["log_scales"][3] = [-1.0, -2.0, -3.0]                      # large: split
    acc[:] = [0.0, 0.0, 0.01, 0.01, 0.0]
    cnt[:] = [1, 1, 1, 1, 0]                                     # 2 clone, 3 split, 0 and 4 kept
    m = {k: np.full_like(v, 7.0) for k, v in P.items()}
    noise = np.zeros((5, 2, 3), np.float32)
    noise[3, 0] = [1, 0, 0]
    noise[3, 1] = [0, -1, 0]
    o = orc.densify(P, m, m, acc, cnt, noise, extent=4.0)
    assert list(o["kind"]) == [1, 0, 2, 3, 1] and o["n_out"] == 6      # sources 0, 2, 4 | 2 | 3, 3
    out_feat = o["params"]["feat"]
    assert out_feat.shape[0] == 6
    assert np.array_equal(out_feat[:4], P["feat"][[0, 2, 4, 2]]) and np.array_equal(out_feat[4:], P["feat"][[3, 3]])
    assert np.all(o["m"]["feat"][:3] == 7.0) and np.all(o["m"]["feat"][3:] == 0.0)
    q = P["quats"][3].astype(np.float64)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    mu = P["means"][3].astype(np.float64)
    assert np.abs(o["params"]["means"][4] - (mu + np.exp(-1.0) * R[:, 0])).max() < 1e-12
    assert np.abs(o["params"]["means"][5] - (mu - np.exp(-2.0) * R[:, 1])).max() < 1e-12
    assert np.abs(o["params"]["log_scales"][4] - (P["log_scales"][3] - np.log(1.6))).max() < 1e-12
