"""GPU parity of projection, binning, compositing and its backward against the
FP64 oracle, through the C ABI (marked gpu)."""
import math

import numpy as np
import pytest
import torch

from paper_2511_16144_gb300 import synth
from tests.gpu_util import bf16_round, bf16_scene, grad_close, robust_mask

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lgs():
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    from paper_2511_16144_gb300 import build, lgs as L
    build.build()
    L.load()
    return L


def _dev(scene, chan=torch.float32):
    from paper_2511_16144_gb300.render import DeviceScene
    return DeviceScene.from_host(scene, chan_dtype=chan)


def _frame(scene, cams, bg=(0.0, 0.0, 0.0), chan=torch.float32, **kw):
    from paper_2511_16144_gb300.render import Frame
    return Frame(_dev(scene, chan), cams, bg, want_count=True, **kw)


def _np(t):
    return t.detach().cpu().numpy()


# ---------------------------------------------------------------- projection

def test_project_matches_oracle(lgs, oracle_lib):
    scene, cams = synth.tiny()
    ds = _dev(scene)
    proj, rect = lgs.gs_project(*ds.params(), cams)
    proj, rect = _np(proj), _np(rect).astype(np.int32) & 0xFFFF
    o = oracle_lib.project(scene, cams[0])
    valid = o["valid"] == 1
    gvalid = (rect[:, 2] > rect[:, 0]) & (rect[:, 3] > rect[:, 1])
    assert valid.sum() > 500
    # exact rect agreement away from pixel-boundary ties of the support radius
    u, v, r = o["mean2d"][:, 0], o["mean2d"][:, 1], o["radius"]
    edges = np.stack([u - r - 0.5, u + r - 0.5, v - r - 0.5, v + r - 0.5], 1)
    near = (np.abs(edges - np.round(edges)) < 1e-3).any(1)
    sure = ~near
    np.testing.assert_array_equal(gvalid[sure], valid[sure])
    np.testing.assert_array_equal(rect[sure & valid], o["rect"][sure & valid])
    m = valid & gvalid
    np.testing.assert_allclose(proj[m, 0:2], o["mean2d"][m], rtol=0, atol=2e-4)
    np.testing.assert_allclose(proj[m, 6], o["depth"][m], rtol=1e-6)
    np.testing.assert_allclose(proj[m, 5], o["opacity"][m], rtol=0, atol=1e-6)
    cmax = np.abs(o["conic"][m]).max(1, keepdims=True)
    np.testing.assert_allclose(proj[m, 2:5] / cmax, o["conic"][m] / cmax, rtol=0, atol=2e-5)
    assert np.all(proj[~gvalid] == 0)


# ---------------------------------------------------------------- binning

def _bin_inputs(n, ncams, tx, ty, seed, tie_frac=0.1, empty=False, max_extent=6):
    """Seeded rects and depths with projected records whose ellipses reach
    part of each rect (the tile test decides which tiles are binned)."""
    rng = np.random.default_rng(seed)
    rect, depth = synth.synthetic_projected(rng, n, ncams, tx, ty, max_extent=max_extent,
                                            tie_frac=tie_frac)
    if empty:
        rect[:, 2] = rect[:, 0]
    proj = synth.synthetic_records(rng, rect, depth)
    return rect, depth, proj


@pytest.mark.parametrize("n,ncams,tx,ty,seed,ext", [
    (1, 1, 1, 1, 0, 6), (1000, 1, 8, 6, 1, 6), (5000, 3, 13, 7, 2, 6), (20000, 8, 40, 30, 3, 6),
    (70000, 2, 75, 43, 4, 6), (3, 16, 2, 2, 5, 6),
    # rects up to 40 x 40 tiles: one splat's pairs span several rounds of a block
    (4000, 2, 60, 40, 7, 40),
    # 34,000 tiles per camera: no per-block shared-memory tables, global atomics
    (3000, 1, 200, 170, 6, 12)])
def test_bin_sort_bit_exact(lgs, oracle_lib, n, ncams, tx, ty, seed, ext):
    rect, depth, proj = _bin_inputs(n, ncams, tx, ty, seed, max_extent=ext)
    ref = oracle_lib.bin_sort(rect, depth, n, ncams, tx, ty, proj=proj)
    k = len(ref["ids"])
    if n > 100:  # the tile test drops part of the rects' tiles
        area = ((rect[:, 2] - rect[:, 0]) * (rect[:, 3] - rect[:, 1])).sum()
        assert 0 < k < area
    for cap in (k, k + 4099):
        bufs = lgs.BinBuffers(n, ncams, tx, ty, cap, "cuda", want_keys=True)
        lgs.gs_bin_sort(torch.from_numpy(proj).cuda(), torch.from_numpy(rect.astype(np.int16)).cuda(),
                        bufs)
        torch.cuda.synchronize()
        assert int(bufs.k_dev.item()) == k
        np.testing.assert_array_equal(_np(bufs.ids)[:k].view(np.uint32), ref["ids"])
        np.testing.assert_array_equal(_np(bufs.keys)[:k].view(np.uint64), ref["keys"])
        np.testing.assert_array_equal(_np(bufs.ranges).view(np.uint32), ref["ranges"])


@pytest.mark.parametrize("tie_frac", [0.0, 0.1])
def test_bin_sort_long_segments_bit_exact(lgs, oracle_lib, tie_frac):
    """Tiles at every size tier of the per-tile sort: exactly 2,048 (the last
    of the eight-keys-a-thread blocks), 2,049 and 3,000 (sixteen keys a
    thread), 5,000 and exactly 12,288 (the 1024-thread blocks' shared-memory
    limit), 12,289 and 30,000 (chunk by chunk from global memory), all in
    the third camera, next to two cameras of ordinary tiles; with and without
    equal depths."""
    rng = np.random.default_rng(31)
    ncams, tx, ty, n = 3, 9, 7, 70000
    rect, depth = synth.synthetic_projected(rng, n, ncams, tx, ty, max_extent=3,
                                            tie_frac=tie_frac)
    sizes = [(0, 5000), (3, 12288), (10, 12289), (40, 30000), (20, 3000), (25, 2048),
             (30, 2049)]  # (tile, instances)
    rect[2 * n:] = 0  # camera 2: only the long tiles
    proj = synth.synthetic_records(rng, rect, depth)
    i0 = 2 * n
    for t, cnt in sizes:
        x, y = t % tx, t // tx
        rect[i0:i0 + cnt] = [x, y, x + 1, y + 1]
        proj[i0:i0 + cnt, 0:2] = [16 * x + 8, 16 * y + 8]  # the mean inside: always reached
        i0 += cnt
    ref = oracle_lib.bin_sort(rect, depth, n, ncams, tx, ty, proj=proj)
    k = len(ref["ids"])
    counts = (ref["ranges"][:, 1] - ref["ranges"][:, 0]).reshape(ncams, -1)
    assert [int(counts[2, t]) for t, _ in sizes] == [c for _, c in sizes]
    bufs = lgs.BinBuffers(n, ncams, tx, ty, k, "cuda", want_keys=True)
    for _ in range(2):  # the second call reuses the workspace
        lgs.gs_bin_sort(torch.from_numpy(proj).cuda(),
                        torch.from_numpy(rect.astype(np.int16)).cuda(), bufs)
        torch.cuda.synchronize()
        assert int(bufs.k_dev.item()) == k
        np.testing.assert_array_equal(_np(bufs.ids)[:k].view(np.uint32), ref["ids"])
        np.testing.assert_array_equal(_np(bufs.keys)[:k].view(np.uint64), ref["keys"])
        np.testing.assert_array_equal(_np(bufs.ranges).view(np.uint32), ref["ranges"])


def test_bin_sort_huge_rects_bit_exact(lgs, oracle_lib):
    """Rects of over 2^20 tiles (one camera of 1100 x 1000 tiles): their pairs
    span thousands of rounds of a block and their tile coordinates come from
    the exact integer division; next to a rect just under 2^20 tiles (the
    reciprocal path), one of exactly 32 tiles (the largest with a hit mask),
    one of 33, and a one-tile rect."""
    ncams, tx, ty = 1, 1100, 1000
    rect = np.array([[0, 0, 1100, 1000], [100, 50, 1100, 1000], [10, 10, 18, 14],
                     [20, 20, 31, 23], [5, 5, 6, 6]], dtype=np.int32)
    n = rect.shape[0]
    depth = np.array([3.0, 2.0, 1.0, 1.5, 0.5], np.float32)
    rng = np.random.default_rng(77)
    proj = synth.synthetic_records(rng, rect, depth)
    # wide isotropic ellipses for the two big rects: they reach most of their tiles
    for i, (u, v, s) in enumerate([(8800.0, 8000.0, 4000.0), (9000.0, 8300.0, 2500.0)]):
        o = 0.9
        proj[i, 0:6] = [u, v, 1.0 / s ** 2, 0.0, 1.0 / s ** 2, o]
        proj[i, 7] = 2.0 * np.log(255.0 * o) * 1.001 + 0.01
    ref = oracle_lib.bin_sort(rect, depth, n, ncams, tx, ty, proj=proj)
    k = len(ref["ids"])
    assert k > (1 << 20)
    bufs = lgs.BinBuffers(n, ncams, tx, ty, k, "cuda", want_keys=True)
    lgs.gs_bin_sort(torch.from_numpy(proj).cuda(), torch.from_numpy(rect.astype(np.int16)).cuda(),
                    bufs)
    torch.cuda.synchronize()
    assert int(bufs.k_dev.item()) == k
    np.testing.assert_array_equal(_np(bufs.ids)[:k].view(np.uint32), ref["ids"])
    np.testing.assert_array_equal(_np(bufs.keys)[:k].view(np.uint64), ref["keys"])
    np.testing.assert_array_equal(_np(bufs.ranges).view(np.uint32), ref["ranges"])


def test_bin_sort_empty_and_overflow(lgs, oracle_lib):
    n, ncams, tx, ty = 4000, 2, 20, 10
    rect, depth, proj = _bin_inputs(n, ncams, tx, ty, 11, empty=True)
    bufs = lgs.BinBuffers(n, ncams, tx, ty, 16, "cuda")
    lgs.gs_bin_sort(torch.from_numpy(proj).cuda(), torch.from_numpy(rect.astype(np.int16)).cuda(),
                    bufs)
    torch.cuda.synchronize()
    assert int(bufs.k_dev.item()) == 0
    assert int(_np(bufs.ranges).sum()) == 0
    # capacity one short of K: K is still reported, nothing is sorted
    rect, depth, proj = _bin_inputs(n, ncams, tx, ty, 12)
    k = len(oracle_lib.bin_sort(rect, depth, n, ncams, tx, ty, proj=proj)["ids"])
    bufs = lgs.BinBuffers(n, ncams, tx, ty, k - 1, "cuda")
    bufs.ranges.fill_(7)
    lgs.gs_bin_sort(torch.from_numpy(proj).cuda(), torch.from_numpy(rect.astype(np.int16)).cuda(),
                    bufs)
    torch.cuda.synchronize()
    assert int(bufs.k_dev.item()) == k
    assert int(_np(bufs.ranges).sum()) == 0


def test_bin_sort_invalid_arguments(lgs):
    bufs = lgs.BinBuffers(10, 1, 2, 2, 64, "cuda")
    proj = torch.zeros((10, 8), device="cuda")
    rect = torch.zeros((10, 4), dtype=torch.int16, device="cuda")
    bufs.workspace_bytes = 8  # too small
    with pytest.raises(lgs.LgsError, match="workspace"):
        lgs.gs_bin_sort(proj, rect, bufs)


# ---------------------------------------------------------------- forward

def _check_maps(out, o, keep, atol=1e-5):
    """Strict parity on pixels whose decisions are robust; on the few pixels
    where an FP32 skip / clamp / stop decision may flip, the difference must
    stay within what one flipped decision can cause (a blend weight of at
    most 2/255 of a unit-range channel, or one stop-level blend)."""
    frac = 1.0 - keep.mean()
    assert frac < 1e-2, f"{frac:.2e} of pixels within the decision margin"
    dscale = max(1.0, np.abs(o["depth"]).max())
    fscale = max(1.0, np.abs(o["feat"]).max()) if o["feat"].size else 1.0
    for k, scale in (("rgb", 1.0), ("feat", 1.0), ("T_final", 1.0), ("depth", dscale)):
        d = np.abs(out[k] - o[k])
        assert d[keep].max() <= atol * scale, (k, d[keep].max())
        if (~keep).any():
            bound = 2.0 / 255.0 * (dscale if k == "depth" else fscale if k == "feat" else 1.0)
            assert d[~keep].max() <= bound, (k, "flagged", d[~keep].max())
    np.testing.assert_array_equal(out["n_contrib"][keep], o["n_contrib"][keep])


def _compare_forward(fr, o, keep, cam_index=0, atol=1e-5):
    out = {k: _np(v[cam_index]) for k, v in fr.out.items() if v is not None}
    _check_maps(out, o, keep, atol)
    return out


@pytest.mark.parametrize("chan", ["f32", "bf16"])
def test_render_fwd_tiny_matches_oracle(lgs, oracle_lib, chan):
    scene, cams = synth.tiny()
    bg = (0.1, 0.2, 0.3)
    tch = torch.float32 if chan == "f32" else torch.bfloat16
    fr = _frame(scene, cams, bg, chan=tch)
    ref = scene if chan == "f32" else bf16_scene(scene)
    o = oracle_lib.render(ref, cams[0], bg=bg)
    _compare_forward(fr, o, robust_mask(o))
    if chan == "bf16":
        # quantisation error of BF16 channels against the unrounded FP64 render
        o32 = oracle_lib.render(scene, cams[0], bg=bg)
        q = np.abs(_np(fr.out["feat"][0]) - o32["feat"]).max()
        assert q < 2e-2


def test_render_fwd_ragged_and_empty(lgs, oracle_lib):
    # 37x29 image: partial tiles on both edges; plus a scene with nothing visible
    scene, _ = synth.tiny()
    cam = synth.Camera(40.0, 40.0, 18.5, 14.5, 37, 29, synth.identity_view())
    fr = _frame(scene, [cam], (0.5, 0.25, 0.0))
    o = oracle_lib.render(scene, cam, bg=(0.5, 0.25, 0.0))
    _compare_forward(fr, o, robust_mask(o))
    behind = synth.Scene(scene.means * np.array([1, 1, -1], np.float32), scene.quats,
                         scene.log_scales, scene.opacity_logits, scene.colors, scene.feats)
    fr = _frame(behind, [cam], (0.5, 0.25, 0.0))
    assert fr.k == 0
    np.testing.assert_array_equal(_np(fr.out["rgb"][0]), np.broadcast_to([0.5, 0.25, 0.0], (29, 37, 3)))
    assert np.all(_np(fr.out["T_final"]) == 1.0) and np.all(_np(fr.out["n_contrib"]) == 0)


def test_render_fwd_multi_camera(lgs, oracle_lib):
    scene, cams = synth.small_window(n=500, size=32, n_cams=3)
    fr = _frame(scene, cams, (0.0, 0.0, 0.0))
    for c in range(3):
        o = oracle_lib.render(scene, cams[c])
        _compare_forward(fr, o, robust_mask(o), cam_index=c)


def test_render_fwd_indoor_full_size_crop(lgs, oracle_lib):
    """Full 300k-Gaussian 640x480 frame on the GPU; oracle on the 64x64
    centre crop (FP32 and BF16 channels)."""
    scene, cams = synth.indoor()
    crop = (288, 208, 64, 64)
    for chan in (torch.float32, torch.bfloat16):
        fr = _frame(scene, cams, chan=chan)
        ref = scene if chan == torch.float32 else bf16_scene(scene)
        o = oracle_lib.render(ref, cams[0], crop=crop)
        x0, y0, w, h = crop
        keep = robust_mask(o)
        out = {k: _np(v[0])[y0:y0 + h, x0:x0 + w] for k, v in fr.out.items() if v is not None}
        _check_maps(out, o, keep)
        assert o["n_contrib"].mean() > 5


def test_render_fwd_plain_512(lgs, oracle_lib):
    """The plain path: 512 feature channels in 16 chunks of 32."""
    scene, cams = synth.embedding_scene(n=30000)
    cam = synth.Camera(131.25, 131.25, 80.0, 60.0, 160, 120, cams[0].viewmat)
    fr = _frame(scene, [cam])
    o = oracle_lib.render(scene, cam)
    _compare_forward(fr, o, robust_mask(o))


# ---------------------------------------------------------------- backward

def _upstream(shape_hw, d, keep, seed):
    rng = np.random.default_rng(seed)
    h, w = shape_hw
    g = [rng.standard_normal((h, w, 3)) * keep[..., None], rng.standard_normal((h, w)) * keep,
         rng.standard_normal((h, w, d)) * keep[..., None]]
    return [x.astype(np.float32) for x in g]


def _gpu_grads(fr, gs):
    t = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in gs]
    if t[0].dim() == 3:
        t = [x.unsqueeze(0) for x in t]
    return {k: _np(v) for k, v in fr.backward(*t).items()}


@pytest.mark.parametrize("which,chan", [("tiny", "f32"), ("window", "f32"), ("tiny", "bf16")])
def test_render_bwd_matches_oracle(lgs, oracle_lib, which, chan):
    if which == "tiny":
        scene, cams = synth.tiny()
    else:
        scene, cams = synth.small_window(n=500, size=32)
    bg = (0.1, 0.2, 0.3)
    tch = torch.float32 if chan == "f32" else torch.bfloat16
    fr = _frame(scene, cams, bg, chan=tch)
    ref = scene if chan == "f32" else bf16_scene(scene)
    o = oracle_lib.render(ref, cams[0], bg=bg)
    keep = robust_mask(o, 1e-3)
    g = _upstream(o["depth"].shape, scene.feats.shape[1], keep, 7)
    gg = _gpu_grads(fr, g)
    go = oracle_lib.render_backward(ref, cams[0], *g, bg=bg)
    # raster part: per-Gaussian 2D gradients before the projection chain rule
    g2 = _np(fr.grad2d)[:, :7]
    grad_close(g2, go["proj"], name="grad2d")
    for k in ("colors", "feats", "opacity_logits", "means", "log_scales", "quats"):
        grad_close(gg[k], go[k], name=k)


def test_render_bwd_multi_camera_is_sum(lgs, oracle_lib):
    scene, cams = synth.small_window(n=500, size=32, n_cams=3)
    fr = _frame(scene, cams)
    gs, acc = [], None
    for c in range(3):
        o = oracle_lib.render(scene, cams[c])
        g = _upstream(o["depth"].shape, 16, robust_mask(o, 1e-3), 20 + c)
        gs.append(g)
        go = oracle_lib.render_backward(scene, cams[c], *g)
        acc = go if acc is None else {k: acc[k] + go[k] for k in acc}
    batched = [np.stack([g[i] for g in gs]) for i in range(3)]
    gg = _gpu_grads(fr, batched)
    for k in ("colors", "feats", "opacity_logits", "means", "log_scales", "quats"):
        grad_close(gg[k], acc[k], name=k)


def test_render_bwd_indoor_full_size_crop(lgs, oracle_lib):
    """Full 640x480 frame over 300k Gaussians; upstream gradient only on the
    64x64 centre crop, so the oracle's crop backward is the whole answer."""
    scene, cams = synth.indoor()
    crop = (288, 208, 64, 64)
    fr = _frame(scene, cams)
    o = oracle_lib.render(scene, cams[0], crop=crop)
    keep = robust_mask(o, 1e-3)
    g = _upstream(o["depth"].shape, 16, keep, 3)
    full = [np.zeros((480, 640, 3), np.float32), np.zeros((480, 640), np.float32),
            np.zeros((480, 640, 16), np.float32)]
    x0, y0, w, h = crop
    for f, part in zip(full, g):
        f[y0:y0 + h, x0:x0 + w] = part
    gg = _gpu_grads(fr, full)
    go = oracle_lib.render_backward(scene, cams[0], *g, crop=crop)
    for k in ("colors", "feats", "opacity_logits", "means", "log_scales", "quats"):
        grad_close(gg[k], go[k], name=k)


def test_render_bwd_plain_512(lgs, oracle_lib):
    scene, cams = synth.embedding_scene(n=20000)
    cam = synth.Camera(131.25, 131.25, 80.0, 60.0, 160, 120, cams[0].viewmat)
    fr = _frame(scene, [cam])
    crop = (48, 36, 40, 32)
    o = oracle_lib.render(scene, cam, crop=crop)
    keep = robust_mask(o, 1e-3)
    g = _upstream(o["depth"].shape, 512, keep, 5)
    full = [np.zeros((120, 160, 3), np.float32), np.zeros((120, 160), np.float32),
            np.zeros((120, 160, 512), np.float32)]
    x0, y0, w, h = crop
    for f, part in zip(full, g):
        f[y0:y0 + h, x0:x0 + w] = part
    gg = _gpu_grads(fr, full)
    go = oracle_lib.render_backward(scene, cam, *g, crop=crop)
    for k in ("colors", "feats", "opacity_logits", "means", "log_scales", "quats"):
        grad_close(gg[k], go[k], name=k)


def test_autograd_function_matches_direct_backward(lgs):
    from paper_2511_16144_gb300.render import DeviceScene, Frame, render
    scene, cams = synth.small_window(n=300, size=32, n_cams=2)
    ds = DeviceScene.from_host(scene)
    leaves = [t.clone().requires_grad_(True) for t in
              (ds.means, ds.quats, ds.log_scales, ds.opacity_logits, ds.colors, ds.feats)]
    rgb, dep, feat = render(DeviceScene(*leaves), cams)
    gen = torch.Generator(device="cuda").manual_seed(0)
    w = [torch.randn(x.shape, device="cuda", generator=gen) for x in (rgb, dep, feat)]
    loss = sum((a * b).sum() for a, b in zip((rgb, dep, feat), w))
    loss.backward()
    fr = Frame(ds, cams)
    direct = fr.backward(*w)
    for leaf, k in zip(leaves, ("means", "quats", "log_scales", "opacity_logits", "colors", "feats")):
        # the two runs differ only in the order of float atomics
        scale = direct[k].abs().max().item()
        torch.testing.assert_close(leaf.grad, direct[k], rtol=1e-4, atol=1e-5 * scale)


def test_l1_loss_matches_oracle(lgs, oracle_lib):
    rng = np.random.default_rng(1)
    pred = rng.standard_normal(100003).astype(np.float32)
    tgt = rng.standard_normal(100003).astype(np.float32)
    tgt[:10] = pred[:10]  # exact ties give sign 0
    for dt in (torch.float32, torch.bfloat16):
        t_dev = torch.from_numpy(tgt).cuda().to(dt)
        t_ref = bf16_round(tgt) if dt == torch.bfloat16 else tgt
        grad = torch.empty(pred.size, device="cuda")
        loss = torch.zeros(1, device="cuda")
        lgs.lgs_l1_loss(torch.from_numpy(pred).cuda(), t_dev, 0.1, grad, loss)
        l_ref, g_ref = oracle_lib.l1_loss_grad(pred, t_ref, 0.1)
        assert abs(loss.item() - l_ref) <= 1e-5 * l_ref
        np.testing.assert_allclose(_np(grad), g_ref, rtol=1e-6, atol=0)


# ---------------------------------------------------------------- full-size windows

def _crop_parity(fr, scene, cam, cam_index, crop, chan_scene=None):
    from oracle import render as orender
    o = orender(chan_scene or scene, cam, crop=crop)
    x0, y0, w, h = crop
    out = {k: _np(v[cam_index])[y0:y0 + h, x0:x0 + w] for k, v in fr.out.items() if v is not None}
    _check_maps(out, o, robust_mask(o))
    return o


def _crop_backward(fr, scene, cams, cam_index, crop, seed, chan_scene=None):
    from oracle import render as orender, render_backward
    ref = chan_scene or scene
    cam = cams[cam_index]
    o = orender(ref, cam, crop=crop)
    g = _upstream(o["depth"].shape, scene.feats.shape[1], robust_mask(o, 1e-3), seed)
    C, H, W = len(cams), cam.height, cam.width
    full = [np.zeros((C, H, W, 3), np.float32), np.zeros((C, H, W), np.float32),
            np.zeros((C, H, W, scene.feats.shape[1]), np.float32)]
    x0, y0, w, h = crop
    for f, part in zip(full, g):
        f[cam_index, y0:y0 + h, x0:x0 + w] = part
    gg = _gpu_grads(fr, full)
    go = render_backward(ref, cam, *g, crop=crop)
    for k in ("colors", "feats", "opacity_logits", "means", "log_scales", "quats"):
        grad_close(gg[k], go[k], name=k)


def test_render_window8_full_size(lgs, oracle_lib):
    """The differentiable mapping window: 8 keyframes of 640x480 over 300k
    Gaussians in one launch; sampled crops of three cameras forward, and the
    backward of an upstream gradient on one crop of one camera."""
    scene, cams = synth.indoor(n_cams=8)
    fr = _frame(scene, cams)
    assert fr.k > 8 * 10 ** 6
    for c, crop in ((0, (300, 220, 40, 40)), (3, (0, 0, 40, 40)), (7, (600, 440, 40, 40))):
        _crop_parity(fr, scene, cams[c], c, crop)
    _crop_backward(fr, scene, cams, 5, (280, 200, 48, 48), 11)


def test_render_outdoor_full_size(lgs, oracle_lib):
    """Large outdoor scale: 2M Gaussians in 40x40x8 m, 8 keyframes of
    1200x680 (a partial bottom tile row), BF16 channels; sampled crops
    forward (including the partial row) and one crop backward."""
    scene, cams = synth.outdoor()
    fr = _frame(scene, cams, chan=torch.bfloat16)
    ref = bf16_scene(scene)
    for c, crop in ((0, (584, 324, 32, 32)), (6, (1168, 648, 32, 32))):
        _crop_parity(fr, scene, cams[c], c, crop, chan_scene=ref)
    _crop_backward(fr, scene, cams, 2, (600, 300, 32, 32), 12, chan_scene=ref)
