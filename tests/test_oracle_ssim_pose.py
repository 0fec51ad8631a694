"""Pins of the D-SSIM oracle (Sec. III-B.3's photometric loss) and of the
camera pose gradient (Sec. III-B.2's keyframe pose refinement)."""
import math

import numpy as np
import pytest

import oracle
from oracle import ssim
from paper_2511_16144_gb300 import synth


# ---------------------------------------------------------------- D-SSIM

def test_window_taps():
    g = ssim.window_1d()
    assert g.shape == (11,) and abs(g.sum() - 1) < 1e-15
    np.testing.assert_allclose(g, g[::-1], rtol=0, atol=0)
    # Gaussian of sigma 1.5: neighbouring taps differ by exp((2k+1) / (2 sigma^2))
    for k in range(5):
        assert g[5 + k] / g[6 + k] == pytest.approx(math.exp((2 * k + 1) / (2 * 2.25)), rel=1e-12)


def test_ssim_of_identical_images_is_one():
    rng = np.random.default_rng(0)
    x = rng.random((14, 17, 3))
    np.testing.assert_allclose(ssim.ssim_map(x, x), 1.0, rtol=0, atol=1e-12)
    loss, g = ssim.dssim_loss(x, x)
    assert abs(loss) < 1e-12 and np.abs(g).max() < 1e-12


def test_ssim_of_constant_images_interior():
    a, b = 0.3, 0.7
    x = np.full((30, 30, 3), a)
    y = np.full((30, 30, 3), b)
    m = ssim.ssim_map(x, y)
    expect = (2 * a * b + ssim.C1) / (a * a + b * b + ssim.C1)
    np.testing.assert_allclose(m[5:25, 5:25], expect, rtol=1e-12)


def _brute_ssim(x, y):
    """Direct window sums with explicit zero padding, one pixel at a time."""
    g = ssim.window_1d()
    h, w = x.shape
    out = np.zeros((h, w))
    for i in range(h):
        for j in range(w):
            s = dict(mx=0.0, my=0.0, xx=0.0, yy=0.0, xy=0.0)
            for di in range(-5, 6):
                for dj in range(-5, 6):
                    ii, jj = i + di, j + dj
                    if 0 <= ii < h and 0 <= jj < w:
                        wt = g[di + 5] * g[dj + 5]
                        s["mx"] += wt * x[ii, jj]
                        s["my"] += wt * y[ii, jj]
                        s["xx"] += wt * x[ii, jj] ** 2
                        s["yy"] += wt * y[ii, jj] ** 2
                        s["xy"] += wt * x[ii, jj] * y[ii, jj]
            mx, my = s["mx"], s["my"]
            vx, vy, cxy = s["xx"] - mx * mx, s["yy"] - my * my, s["xy"] - mx * my
            out[i, j] = ((2 * mx * my + 0.0001) * (2 * cxy + 0.0009)
                         / ((mx * mx + my * my + 0.0001) * (vx + vy + 0.0009)))
    return out


def test_ssim_against_window_sums():
    rng = np.random.default_rng(1)
    x, y = rng.random((9, 13, 3)), rng.random((9, 13, 3))
    m = ssim.ssim_map(x, y)
    for ch in range(3):
        np.testing.assert_allclose(m[..., ch], _brute_ssim(x[..., ch], y[..., ch]), rtol=1e-12)


def test_dssim_gradient_finite_differences():
    rng = np.random.default_rng(2)
    x, y = rng.random((2, 10, 12, 3)), rng.random((2, 10, 12, 3))
    loss, g = ssim.dssim_loss(x, y, weight=0.7)
    assert loss == pytest.approx(0.7 * (1 - ssim.ssim_map(x, y).mean()), rel=1e-12)
    eps = 1e-4  # the loss is smooth; larger steps keep FD roundoff below 1e-12
    idx = [tuple(rng.integers(0, s) for s in x.shape) for _ in range(40)]
    idx += [(0, 0, 0, 0), (1, 9, 11, 2), (0, 5, 0, 1)]  # corners and edges
    for k in idx:
        xp, xm = x.copy(), x.copy()
        xp[k] += eps
        xm[k] -= eps
        fd = (ssim.dssim_loss(xp, y, 0.7)[0] - ssim.dssim_loss(xm, y, 0.7)[0]) / (2 * eps)
        assert g[k] == pytest.approx(fd, rel=1e-5, abs=1e-12)


def test_rgb_loss_combines_l1_and_dssim():
    rng = np.random.default_rng(3)
    x, y = rng.random((8, 9, 3)), rng.random((8, 9, 3))
    loss, g = ssim.rgb_loss(x, y)
    ld, gd = ssim.dssim_loss(x, y)
    assert loss == pytest.approx(0.8 * np.abs(x - y).mean() + 0.2 * ld, rel=1e-14)
    np.testing.assert_allclose(g, 0.8 * np.sign(x - y) / x.size + 0.2 * gd, rtol=1e-14)


# ---------------------------------------------------------------- pose gradient

def _rot(axis, ang):
    k = np.asarray(axis, float)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def _perturb(cam, comp, eps):
    """Camera whose world->camera transform is exp(eps e_comp^) T (left)."""
    vm = np.asarray(cam.viewmat, float).reshape(3, 4)
    R, t = vm[:, :3], vm[:, 3]
    if comp < 3:
        t = t + eps * np.eye(3)[comp]
    else:
        Q = _rot(np.eye(3)[comp - 3], eps)
        R, t = Q @ R, Q @ t
    return synth.Camera(cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height,
                        np.concatenate([R, t[:, None]], 1).reshape(-1), cam.znear)


def _linear_loss(scene, cam, g):
    o = oracle.render(scene, cam)
    return float((o["rgb"] * g[0]).sum() + (o["depth"] * g[1]).sum() + (o["feat"] * g[2]).sum())


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_pose_gradient_finite_differences(seed):
    """Central differences of a linear functional of the render under left
    perturbations of the camera, upstream gradients only on pixels whose
    skip / clamp / stop decisions are robust (unchanged by the steps)."""
    scene, cams = synth.small_window(n=60, size=24, seed=1002 + seed)
    cam = cams[0]
    o = oracle.render(scene, cam)
    keep = (o["margin"] > 1e-3) & (o["zgap"] > 1e-6)
    rng = np.random.default_rng(seed)
    h, w = o["depth"].shape
    g = [rng.standard_normal((h, w, 3)) * keep[..., None], rng.standard_normal((h, w)) * keep,
         rng.standard_normal((h, w, scene.feats.shape[1])) * keep[..., None]]
    go = oracle.render_backward(scene, cam, *g)
    pg = oracle.pose_grad(scene, cam, go["proj"])
    eps = 1e-6
    for comp in range(6):
        vals = []
        for sgn in (1, -1):
            cp = _perturb(cam, comp, sgn * eps)
            vals.append(_linear_loss(scene, cp, g))
            assert np.array_equal(oracle.render(scene, cp)["n_contrib"][keep], o["n_contrib"][keep])
        fd = (vals[0] - vals[1]) / (2 * eps)
        scale = max(abs(fd), 1e-2 * np.abs(pg).max())
        assert abs(pg[comp] - fd) <= 2e-4 * scale, (comp, pg[comp], fd)


def test_pose_translation_gradient_is_the_rotated_mean_gradient():
    """Moving the camera by rho moves every Gaussian by -R^T rho, so
    dL/drho = R sum_i dL/dp_i."""
    scene, cams = synth.small_window(n=300, size=24)
    cam = cams[0]
    o = oracle.render(scene, cam)
    rng = np.random.default_rng(9)
    h, w = o["depth"].shape
    g = [rng.standard_normal((h, w, 3)), rng.standard_normal((h, w)),
         rng.standard_normal((h, w, scene.feats.shape[1]))]
    go = oracle.render_backward(scene, cam, *g)
    pg = oracle.pose_grad(scene, cam, go["proj"])
    R = np.asarray(cam.viewmat, float).reshape(3, 4)[:, :3]
    np.testing.assert_allclose(pg[:3], R @ go["means"].sum(0), rtol=1e-9,
                               atol=1e-12 * np.abs(pg[:3]).max())
