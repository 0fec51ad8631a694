"""GPU parity of the D-SSIM loss term (Sec. III-B.3) and of the camera pose
gradient (Sec. III-B.2) against the FP64 oracle, through the C ABI (gpu)."""
import numpy as np
import pytest
import torch

from paper_2511_16144_gb300 import synth
from tests.gpu_util import grad_close, robust_mask
from tests.test_gpu_render import _frame, _np, _upstream

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lgs():
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    from paper_2511_16144_gb300 import build, lgs as L
    build.build()
    L.load()
    return L


def _dssim_gpu(lgs, x, y, weight, grad0=None):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    g = t(grad0) if grad0 is not None else torch.zeros(x.shape, device="cuda")
    loss = torch.zeros(1, device="cuda")
    lgs.lgs_dssim_loss(t(x), t(y), weight, g, loss)
    torch.cuda.synchronize()
    return float(loss.item()), _np(g)


@pytest.mark.parametrize("shape", [(1, 37, 45), (2, 16, 16), (3, 5, 70)])
def test_dssim_matches_oracle(lgs, shape):
    from oracle import ssim
    rng = np.random.default_rng(sum(shape))
    x = rng.random(shape + (3,)).astype(np.float32)
    y = np.clip(x + 0.2 * rng.standard_normal(x.shape), 0, 1).astype(np.float32)
    loss, g = _dssim_gpu(lgs, x, y, 0.2)
    lr, gr = ssim.dssim_loss(x, y, 0.2)
    assert loss == pytest.approx(lr, rel=1e-5)
    scale = np.abs(gr).max()
    assert np.linalg.norm(g - gr) <= 1e-4 * np.linalg.norm(gr)
    assert np.abs(g - gr).max() <= 1e-3 * scale
    # accumulates into an existing gradient (the L1 term's)
    g0 = rng.standard_normal(x.shape).astype(np.float32)
    _, g2 = _dssim_gpu(lgs, x, y, 0.2, g0)
    np.testing.assert_allclose(g2 - g0, g, rtol=0, atol=1e-6 * max(1.0, np.abs(g0).max()))


def test_dssim_identical_and_full_frame(lgs):
    from oracle import ssim
    rng = np.random.default_rng(7)
    x = rng.random((1, 480, 640, 3)).astype(np.float32)
    loss, g = _dssim_gpu(lgs, x, x, 1.0)
    assert abs(loss) < 1e-5 and np.abs(g).max() < 1e-9
    y = np.clip(x + 0.1 * rng.standard_normal(x.shape), 0, 1).astype(np.float32)
    loss, g = _dssim_gpu(lgs, x, y, 0.2)
    lr, gr = ssim.dssim_loss(x, y, 0.2)
    assert loss == pytest.approx(lr, rel=1e-4)
    assert np.linalg.norm(g - gr) <= 1e-4 * np.linalg.norm(gr)


def _pose_case(lgs, oracle_lib, scene, cams, seed, crop=None):
    fr = _frame(scene, cams)
    c = len(cams)
    ups, pose_ref = [], []
    for k in range(c):
        o = oracle_lib.render(scene, cams[k], crop=crop)
        keep = robust_mask(o, 1e-3)
        g = _upstream(o["depth"].shape, scene.feats.shape[1], keep, seed + k)
        go = oracle_lib.render_backward(scene, cams[k], *g, crop=crop)
        pose_ref.append(oracle_lib.pose_grad(scene, cams[k], go["proj"]))
        if crop is not None:
            x0, y0, w, h = crop
            full = [np.zeros((cams[k].height, cams[k].width) + a.shape[2:], np.float32)
                    for a in g]
            for f, part in zip(full, g):
                f[y0:y0 + h, x0:x0 + w] = part
            g = full
        ups.append(g)
    batched = [np.stack([u[i] for u in ups]) for i in range(3)]
    t = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in batched]
    fr.backward(*t)
    ds = fr.scene
    dp = lgs.gs_pose_grad(ds.means, ds.quats, ds.log_scales, ds.opacity_logits, cams, fr.grad2d)
    torch.cuda.synchronize()
    return _np(dp), np.stack(pose_ref)


def test_pose_grad_matches_oracle(lgs, oracle_lib):
    scene, cams = synth.small_window(n=500, size=32, n_cams=3)
    got, ref = _pose_case(lgs, oracle_lib, scene, cams, 30)
    for k in range(3):
        grad_close(got[k], ref[k], name=f"pose camera {k}")
    # the translation part is the rotated sum of the mean gradients
    assert np.abs(ref).max() > 0


def test_pose_grad_full_size_crop(lgs, oracle_lib):
    """640x480 frame over 300k Gaussians, upstream gradient on a 64x64 crop."""
    scene, cams = synth.indoor()
    got, ref = _pose_case(lgs, oracle_lib, scene, cams, 40, crop=(288, 208, 64, 64))
    grad_close(got[0], ref[0], name="pose")
