"""Pins of the FP64 oracle's projection, compositing and backward against
closed forms, invariants and finite differences (no GPU).

Each closed form here is derived from the mathematics of EWA splatting and
front-to-back alpha compositing (the "standard 3DGS pipeline" the paper's
Sec. III-B.1 renders with), not from the oracle's code.
"""
import math

import numpy as np
import pytest

from paper_2511_16144_gb300 import synth

ALPHA_MIN, ALPHA_MAX, T_STOP = 1.0 / 255.0, 0.99, 1e-4


def one_scene(means, log_scales, quats=None, logits=None, colors=None, feats=None):
    means = np.asarray(means, np.float32).reshape(-1, 3)
    n = means.shape[0]
    ls = np.asarray(log_scales, np.float32).reshape(n, 3)
    q = np.tile([1, 0, 0, 0], (n, 1)).astype(np.float32) if quats is None else \
        np.asarray(quats, np.float32).reshape(n, 4)
    lg = np.zeros(n, np.float32) if logits is None else np.asarray(logits, np.float32).reshape(n)
    c = np.ones((n, 3), np.float32) if colors is None else np.asarray(colors, np.float32).reshape(n, 3)
    f = np.zeros((n, 4), np.float32) if feats is None else np.asarray(feats, np.float32).reshape(n, -1)
    return synth.Scene(means, q, ls, lg, c, f)


def cam(w=64, h=48, f=50.0, cx=None, cy=None):
    return synth.Camera(f, f, w / 2 if cx is None else cx, h / 2 if cy is None else cy, w, h,
                        synth.identity_view())


def sig(x):
    return 1.0 / (1.0 + math.exp(-float(np.float32(x))))


def f32(x):
    """The value the float32 inputs actually carry."""
    return float(np.float32(x))


def scale(s):
    """Scale after the float32 log-scale round trip."""
    return math.exp(f32(math.log(s)))


# ---------------------------------------------------------------- projection

def test_project_isotropic_on_axis(oracle_lib):
    s, z, f = 0.05, 2.0, 50.0
    sc = one_scene([0, 0, z], [math.log(s)] * 3, logits=[0.7])
    p = oracle_lib.project(sc, cam(f=f))
    var = (f * scale(s) / z) ** 2 + 0.3
    assert p["valid"][0] == 1
    np.testing.assert_allclose(p["mean2d"][0], [32.0, 24.0], rtol=0, atol=1e-12)
    np.testing.assert_allclose(p["cov2d"][0], [var, 0.0, var], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(p["conic"][0], [1 / var, 0.0, 1 / var], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(p["opacity"][0], sig(0.7), rtol=1e-12)
    assert p["depth"][0] == pytest.approx(z, abs=1e-6)


def test_project_frontal_anisotropic(oracle_lib):
    # rotation by theta about the optical axis, scales (s1, s2, s3), on axis:
    # the z column of J vanishes, so Sigma2 = (f/z)^2 R2 diag(s1^2, s2^2) R2^T + 0.3 I
    th, s1, s2, s3, z, f = 0.4, 0.08, 0.02, 0.5, 2.5, 60.0
    q = [math.cos(th / 2), 0, 0, math.sin(th / 2)]
    sc = one_scene([0, 0, z], [math.log(s1), math.log(s2), math.log(s3)], quats=q, logits=[1.0])
    p = oracle_lib.project(sc, cam(f=f))
    s1, s2 = scale(s1), scale(s2)
    qw, qz = f32(q[0]), f32(q[3])
    th = 2 * math.atan2(qz, qw)
    R2 = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    S = (f / z) ** 2 * R2 @ np.diag([s1 ** 2, s2 ** 2]) @ R2.T + 0.3 * np.eye(2)
    np.testing.assert_allclose(p["cov2d"][0], [S[0, 0], S[0, 1], S[1, 1]], rtol=1e-9, atol=1e-12)
    det = S[0, 0] * S[1, 1] - S[0, 1] ** 2
    np.testing.assert_allclose(p["conic"][0], [S[1, 1] / det, -S[0, 1] / det, S[0, 0] / det],
                               rtol=1e-9)


def test_project_off_axis_and_clamp(oracle_lib):
    # isotropic off-axis Gaussian at (x, 0, z): J = [[f/z, 0, -f x/z^2], [0, f/z, 0]],
    # Sigma2 = s^2 J J^T + 0.3 I; beyond 1.15 W the ratio x/z is clamped inside J only.
    f, z, s, w, h = 40.0, 2.0, 0.05, 64, 48
    lim = (1.15 * w - w / 2) / f
    for x in (0.3, 3.0):
        sc = one_scene([x, 0, z], [math.log(s)] * 3, logits=[3.0])
        p = oracle_lib.project(sc, cam(w=w, h=h, f=f))
        xe = f32(x)
        xc = min(xe / z, lim) * z
        j = np.array([[f / z, 0, -f * xc / z ** 2], [0, f / z, 0]])
        S = scale(s) ** 2 * j @ j.T + 0.3 * np.eye(2)
        np.testing.assert_allclose(p["cov2d"][0], [S[0, 0], S[0, 1], S[1, 1]], rtol=1e-9)
        np.testing.assert_allclose(p["mean2d"][0], [f * xe / z + w / 2, h / 2], rtol=1e-12)


def test_project_validity(oracle_lib):
    c = cam()
    # behind znear, below 1/255 opacity, and outside the image: all invalid
    sc = one_scene([[0, 0, 0.1], [0, 0, 2.0], [50.0, 0, 2.0], [0, 0, 2.0]],
                   [[math.log(0.05)] * 3] * 4, logits=[0, math.log(1 / 300), 0, 0])
    p = oracle_lib.project(sc, c)
    assert list(p["valid"]) == [0, 0, 0, 1]


def test_project_radius_bounds_support(oracle_lib):
    # every pixel centre outside the radius has o exp(power) < 1/255
    rng = np.random.default_rng(5)
    scene, cams = synth.tiny()
    p = oracle_lib.project(scene, cams[0])
    for i in np.flatnonzero(p["valid"])[:200]:
        a, b, cc = p["conic"][i]
        u, v = p["mean2d"][i]
        r = p["radius"][i]
        ang = rng.random(64) * 2 * np.pi
        d = (r + 1e-9) * np.stack([np.cos(ang), np.sin(ang)], 1)
        power = -0.5 * (a * d[:, 0] ** 2 + cc * d[:, 1] ** 2) - b * d[:, 0] * d[:, 1]
        assert np.all(p["opacity"][i] * np.exp(power) < ALPHA_MIN)


# ---------------------------------------------------------------- compositing

def test_single_gaussian_at_pixel_centre(oracle_lib):
    f, z = 50.0, 2.0
    c = cam(f=f)
    # mean projecting to the centre of pixel (20, 10): u = 20.5, v = 10.5
    x, y = (20.5 - c.cx) * z / f, (10.5 - c.cy) * z / f
    for logit in (-1.0, 0.5, 6.0):
        col, feat, bg = [0.2, 0.5, 0.9], [0.1, -0.3, 0.7, 0.2], [0.3, 0.1, 0.6]
        sc = one_scene([x, y, z], [math.log(0.04)] * 3, logits=[logit], colors=[col], feats=[feat])
        o = oracle_lib.render(sc, c, bg=bg)
        col, feat = [f32(v) for v in col], [f32(v) for v in feat]
        a = min(ALPHA_MAX, sig(logit))
        np.testing.assert_allclose(o["rgb"][10, 20], a * np.array(col) + (1 - a) * np.array(bg),
                                   rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(o["depth"][10, 20], a * z, rtol=1e-6)
        np.testing.assert_allclose(o["feat"][10, 20], a * np.array(feat), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(o["T_final"][10, 20], 1 - a, rtol=1e-12)
        assert o["n_contrib"][10, 20] == 1


def test_single_gaussian_footprint(oracle_lib):
    # isotropic on-axis Gaussian: alpha(px) = o exp(-|d|^2 / (2 var)) where >= 1/255
    f, z, s, logit = 50.0, 2.0, 0.06, 1.3
    c = cam(f=f)
    sc = one_scene([0, 0, z], [math.log(s)] * 3, logits=[logit], colors=[[1, 1, 1]])
    o = oracle_lib.render(sc, c)
    var = (f * scale(s) / z) ** 2 + 0.3
    ys, xs = np.mgrid[0:c.height, 0:c.width]
    d2 = (xs + 0.5 - c.cx) ** 2 + (ys + 0.5 - c.cy) ** 2
    a = sig(logit) * np.exp(-0.5 * d2 / var)
    a = np.where(a >= ALPHA_MIN, np.minimum(a, ALPHA_MAX), 0.0)
    np.testing.assert_allclose(o["rgb"][..., 0], a, rtol=1e-12, atol=1e-15)
    np.testing.assert_array_equal(o["n_contrib"], (a > 0).astype(np.int32))
    assert (a > 0).sum() > 20 and (a == 0).sum() > 20


def test_two_stacked_gaussians_order(oracle_lib):
    f = 50.0
    c = cam(f=f)
    c1, c2 = [1.0, 0.2, 0.0], [0.0, 0.4, 1.0]
    l1, l2 = 0.3, -0.2
    for near_first in (True, False):
        means = [[0, 0, 1.5], [0, 0, 2.5]] if near_first else [[0, 0, 2.5], [0, 0, 1.5]]
        cols = [c1, c2] if near_first else [c2, c1]
        lgs = [l1, l2] if near_first else [l2, l1]
        sc = one_scene(means, [[math.log(0.05)] * 3] * 2, logits=lgs, colors=cols)
        o = oracle_lib.render(sc, c)
        c1, c2 = [f32(v) for v in c1], [f32(v) for v in c2]
        # pixel (32, 24) has its centre at (32.5, 24.5): d = (-0.5, -0.5)
        v1 = (f * scale(0.05) / 1.5) ** 2 + 0.3
        v2 = (f * scale(0.05) / 2.5) ** 2 + 0.3
        a1 = sig(l1) * math.exp(-0.25 / v1)
        a2 = sig(l2) * math.exp(-0.25 / v2)
        exp = a1 * np.array(c1) + (1 - a1) * a2 * np.array(c2)
        np.testing.assert_allclose(o["rgb"][24, 32], exp, rtol=1e-12)
        np.testing.assert_allclose(o["depth"][24, 32], a1 * 1.5 + (1 - a1) * a2 * 2.5, rtol=1e-6)


def test_early_stop_rule(oracle_lib):
    # identical stacked splats with alpha = 0.95 at the pixel: T goes 1, .05,
    # .0025, 1.25e-4; the 4th would give 6.25e-6 < 1e-4, so it stops with 3 blended.
    f, n = 50.0, 6
    c = cam(f=f)
    z = 1.5 + 0.1 * np.arange(n)
    x, y = (10.5 - c.cx) * z / f, (7.5 - c.cy) * z / f
    logit = math.log(0.95 / 0.05)
    sc = one_scene(np.stack([x, y, z], 1), [[math.log(0.05)] * 3] * n, logits=[logit] * n)
    o = oracle_lib.render(sc, c)
    assert o["n_contrib"][7, 10] == 3
    np.testing.assert_allclose(o["T_final"][7, 10], 0.05 ** 3, rtol=1e-6)
    np.testing.assert_allclose(o["rgb"][7, 10], [1 - 0.05 ** 3] * 3, rtol=1e-6)


def test_invariants_random_scene(oracle_lib):
    scene, cams = synth.tiny()
    sc = scene.with_feats(scene.feats)
    white = synth.Scene(sc.means, sc.quats, sc.log_scales, sc.opacity_logits,
                        np.ones_like(sc.colors), np.ones((sc.n, 1), np.float32))
    o = oracle_lib.render(white, cams[0])
    T = o["T_final"]
    assert T.min() >= T_STOP and T.max() <= 1.0
    # with unit colours and zero background, rgb = sum of weights = 1 - T_final
    np.testing.assert_allclose(o["rgb"][..., 0], 1 - T, rtol=0, atol=1e-12)
    np.testing.assert_allclose(o["feat"][..., 0], 1 - T, rtol=0, atol=1e-12)
    assert (o["n_contrib"] > 0).mean() > 0.5
    # T after n blends is at most (1 - 1/255)^n and at least (1 - 0.99)^n
    n = o["n_contrib"]
    assert np.all(T <= (1 - ALPHA_MIN) ** n + 1e-12)
    assert np.all(T >= 0.01 ** n - 1e-12)


def test_permutation_invariance(oracle_lib):
    scene, cams = synth.tiny()
    perm = np.random.default_rng(3).permutation(scene.n)
    a = oracle_lib.render(scene, cams[0])
    b = oracle_lib.render(scene.subset(perm), cams[0])
    for k in ("rgb", "depth", "feat", "T_final"):
        np.testing.assert_allclose(a[k], b[k], rtol=0, atol=1e-12)
    np.testing.assert_array_equal(a["n_contrib"], b["n_contrib"])


def test_crop_matches_full_frame(oracle_lib):
    scene, cams = synth.tiny()
    full = oracle_lib.render(scene, cams[0])
    part = oracle_lib.render(scene, cams[0], crop=(37, 21, 40, 30))
    np.testing.assert_array_equal(part["rgb"], full["rgb"][21:51, 37:77])
    np.testing.assert_array_equal(part["n_contrib"], full["n_contrib"][21:51, 37:77])


# ---------------------------------------------------------------- backward

def _loss(oracle_lib, sc, c, g, bg=(0.1, 0.2, 0.3)):
    o = oracle_lib.render(sc, c, bg=bg)
    return (np.sum(o["rgb"] * g[0]) + np.sum(o["depth"] * g[1]) + np.sum(o["feat"] * g[2])), o


def test_single_gaussian_opacity_gradient_closed_form(oracle_lib):
    # rgb = alpha(px) c with alpha = o e^power (unclamped, bg 0):
    # dL/dlogit = sum_px (g . c) e^power o (1 - o)
    f, z, s, logit = 50.0, 2.0, 0.06, -0.4
    c = cam(f=f)
    col = np.array([0.3, 0.6, 0.9], np.float32).astype(np.float64)
    sc = one_scene([0, 0, z], [math.log(s)] * 3, logits=[logit], colors=[col])
    rng = np.random.default_rng(0)
    g = rng.standard_normal((c.height, c.width, 3))
    zero1, zero4 = np.zeros((c.height, c.width)), np.zeros((c.height, c.width, 4))
    gr = oracle_lib.render_backward(sc, c, g, zero1, zero4)
    var = (f * scale(s) / z) ** 2 + 0.3
    ys, xs = np.mgrid[0:c.height, 0:c.width]
    e = np.exp(-0.5 * ((xs + 0.5 - c.cx) ** 2 + (ys + 0.5 - c.cy) ** 2) / var)
    o = sig(logit)
    a = o * e
    m = a >= ALPHA_MIN
    exp_logit = np.sum((g @ col) * e * m) * o * (1 - o)
    np.testing.assert_allclose(gr["opacity_logits"][0], exp_logit, rtol=1e-10)
    # colour gradient = sum_px w g
    np.testing.assert_allclose(gr["colors"][0], np.sum(g * (a * m)[..., None], axis=(0, 1)),
                               rtol=1e-10)


@pytest.mark.parametrize("seed", [0, 1])
def test_backward_matches_finite_differences(oracle_lib, seed):
    scene, cams = synth.small_window(n=60, size=24, seed=1002 + seed)
    c = cams[0]
    bg = (0.1, 0.2, 0.3)
    base = oracle_lib.render(scene, c, bg=bg)
    rng = np.random.default_rng(seed)
    keep = (base["margin"] > 1e-3) & (base["zgap"] > 1e-6)  # robust decisions
    g = [rng.standard_normal(base["rgb"].shape) * keep[..., None],
         rng.standard_normal(base["depth"].shape) * keep,
         rng.standard_normal(base["feat"].shape) * keep[..., None]]
    an = oracle_lib.render_backward(scene, c, g[0], g[1], g[2], bg=bg)
    p = oracle_lib.project(scene, c)
    active = np.flatnonzero(np.abs(an["colors"]).sum(1) > 0)
    assert active.size > 10
    checked = 0
    for i in active[:25]:
        for name, arr in (("means", scene.means), ("quats", scene.quats),
                          ("log_scales", scene.log_scales), ("opacity_logits", scene.opacity_logits),
                          ("colors", scene.colors), ("feats", scene.feats)):
            flat = arr.reshape(arr.shape[0], -1)
            for j in range(flat.shape[1]):
                h = 1e-6 * max(1.0, abs(float(flat[i, j])))
                vals = []
                for sgn in (1, -1):
                    arr64 = {k: getattr(scene, k).astype(np.float64).copy() for k in
                             ("means", "quats", "log_scales", "opacity_logits", "colors", "feats")}
                    a = arr64[name].reshape(arr64[name].shape[0], -1)
                    a[i, j] += sgn * h
                    sc2 = synth.Scene(**arr64)
                    L, o2 = _loss(oracle_lib, sc2, c, g, bg)
                    assert np.array_equal(o2["n_contrib"][keep], base["n_contrib"][keep])
                    vals.append(L)
                fd = (vals[0] - vals[1]) / (2 * h)
                ana = an[name].reshape(an[name].shape[0], -1)[i, j]
                scale = max(abs(fd), 1e-2 * np.abs(an[name]).max(), 1e-9)
                assert abs(fd - ana) <= 2e-4 * scale, (name, i, j, fd, ana)
                checked += 1
    assert checked > 300
    assert p["valid"][active].all()


def test_backward_linear_in_upstream_gradient(oracle_lib):
    scene, cams = synth.small_window(n=80, size=20)
    c = cams[0]
    rng = np.random.default_rng(9)
    shp = (c.height, c.width)
    g1 = [rng.standard_normal(shp + (3,)), rng.standard_normal(shp), rng.standard_normal(shp + (16,))]
    g2 = [rng.standard_normal(shp + (3,)), rng.standard_normal(shp), rng.standard_normal(shp + (16,))]
    a = oracle_lib.render_backward(scene, c, *g1)
    b = oracle_lib.render_backward(scene, c, *g2)
    s = oracle_lib.render_backward(scene, c, *[x + y for x, y in zip(g1, g2)])
    for k in ("means", "quats", "log_scales", "opacity_logits", "colors", "feats"):
        np.testing.assert_allclose(s[k], a[k] + b[k], rtol=1e-9,
                                   atol=1e-12 * max(1.0, np.abs(s[k]).max()))


def test_projection_backward_finite_differences(oracle_lib):
    # chain rule from random 2D gradients (u, v, conic, opacity, depth) to the
    # parameters, including a Gaussian beyond the J clamp
    scene, cams = synth.small_window(n=12, size=32)
    means = scene.means.copy()
    means[0] = [1.6, 0.3, 1.8]     # x/z beyond the clamp limit in x
    means[1] = [-0.2, -1.4, 2.0]   # beyond the clamp in y
    ls = scene.log_scales.copy()
    ls[:2] = math.log(0.4)         # large enough to reach into the image
    scene = synth.Scene(means, scene.quats, ls, scene.opacity_logits,
                        scene.colors, scene.feats)
    c = cams[0]
    rng = np.random.default_rng(4)
    dp = rng.standard_normal((scene.n, 7))
    an = oracle_lib.project_backward(scene, c, dp)

    def fun(sc):
        p = oracle_lib.project(sc, c)
        vec = np.concatenate([p["mean2d"], p["conic"], p["opacity"][:, None],
                              p["depth"][:, None]], 1)
        return np.sum(vec * dp * p["valid"][:, None])

    base = oracle_lib.project(scene, c)
    assert base["valid"][:2].all()
    for name in ("means", "quats", "log_scales", "opacity_logits"):
        for i in range(scene.n):
            if not base["valid"][i]:
                continue
            arr = getattr(scene, name).astype(np.float64)
            flat = arr.reshape(scene.n, -1)
            for j in range(flat.shape[1]):
                h = 1e-6 * max(1.0, abs(flat[i, j]))
                vals = []
                for sgn in (1, -1):
                    a2 = arr.copy().reshape(scene.n, -1)
                    a2[i, j] += sgn * h
                    kw = {k: getattr(scene, k).astype(np.float64) for k in
                          ("means", "quats", "log_scales", "opacity_logits", "colors", "feats")}
                    kw[name] = a2.reshape(arr.shape)
                    vals.append(fun(synth.Scene(**kw)))
                fd = (vals[0] - vals[1]) / (2 * h)
                ana = an[name].reshape(scene.n, -1)[i, j]
                assert abs(fd - ana) <= 1e-5 * max(abs(fd), 1.0), (name, i, j, fd, ana)
