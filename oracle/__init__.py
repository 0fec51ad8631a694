"""FP64 CPU oracle for the language-feature Gaussian-splatting hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (``paper_2511_16144_gb300``) never imports it, and it
imports nothing from the product package: the two share no code.

Contents
--------
* ``lgs_oracle.c`` (built here into ``liblgs_oracle.so`` with gcc + OpenMP):
  projection, brute-force per-pixel compositing over all Gaussians (no tiles),
  the analytic backward, and the stable-sort binning definition.  The paper
  (LEGO-SLAM, Sec. III-B.1) defers the rasteriser to "the standard 3DGS
  pipeline"; the C file's header lists the textbook definition it writes out.
* ``prune_oracle.c`` (same library): language-guided pruning (Sec. III-C,
  Eq. 4) with the geometric criteria, by brute-force neighbour search; its
  mask decisions are taken in FP32 with a fixed operation order (they turn
  float comparisons into bits), everything else here is float64.
* ``ssim.py``: the D-SSIM term of the photometric loss (Sec. III-B.3) in
  numpy float64.
* ``ae.py``: the scene-adaptive autoencoder (Sec. III-B.3 Eq. 2, Sec. III-B.4
  Eq. 3, Sec. IV-A.2 pretraining) in numpy float64.
* ``losses``: the L1 terms of Eq. 1.

Every float input is converted to float64 before use; integer outputs are
exact.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lgs_oracle.c")
_SRCS = (_SRC, os.path.join(_HERE, "prune_oracle.c"))
_SO = os.path.join(_HERE, "liblgs_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, -O2, OpenMP).  Idempotent."""
    if (not force and os.path.exists(_SO)
            and all(os.path.getmtime(_SO) >= os.path.getmtime(f) for f in _SRCS)):
        return _SO
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC",
                           "-shared", "-o", tmp, *_SRCS, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_SO)
    P = ctypes.c_void_p
    I64, I32 = ctypes.c_int64, ctypes.c_int
    lib.lgso_project.argtypes = [I64, P, P, P, P, P, P, P, P, P, P, P, P, P]
    lib.lgso_render_fwd.argtypes = [I64, I32, P, P, P, P, P, P, P, P, I32, I32, I32, I32,
                                    P, P, P, P, P, P, P]
    lib.lgso_render_bwd.argtypes = [I64, I32, P, P, P, P, P, P, P, P, I32, I32, I32, I32,
                                    P, P, P, P, P, P, P, P, P, P]
    lib.lgso_project_bwd.argtypes = [I64, P, P, P, P, P, P, P, P, P, P]
    lib.lgso_bin_count.argtypes = [I64, I32, P, P]
    lib.lgso_bin_count.restype = I64
    lib.lgso_bin_sort.argtypes = [I64, I32, I32, I32, P, P, P, P, P, P]
    lib.lgso_num_threads.restype = I32
    lib.lgso_pose_grad.argtypes = [I64, P, P, P, P, P, P, P]
    F32 = ctypes.c_float
    lib.lgso_prune.argtypes = [I64, I32, P, P, P, P, I32, F32, F32, F32, F32, P]
    lib.lgso_prune_sample.argtypes = [I64, I32, P, P, P, P, I32, F32, F32, F32, F32, P, I64, P]
    _lib = lib
    return lib


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    """OpenMP threads the oracle uses."""
    return int(_load().lgso_num_threads())


def camera_array(cam) -> np.ndarray:
    """Packs a camera (fx, fy, cx, cy, width, height, znear, viewmat[3,4]) into
    the oracle's double[19] layout."""
    vm = np.asarray(cam.viewmat, dtype=np.float64).reshape(3, 4)
    return np.concatenate([[cam.fx, cam.fy, cam.cx, cam.cy, cam.width, cam.height, cam.znear],
                           vm[:, :3].reshape(-1), vm[:, 3]]).astype(np.float64)


def project(scene, cam) -> dict:
    """EWA projection of every Gaussian for one camera (float64)."""
    lib = _load()
    n = scene.means.shape[0]
    means, quats, ls, lg = (_f64(scene.means), _f64(scene.quats), _f64(scene.log_scales),
                            _f64(scene.opacity_logits))
    out = dict(mean2d=np.zeros((n, 2)), depth=np.zeros(n), conic=np.zeros((n, 3)),
               opacity=np.zeros(n), cov2d=np.zeros((n, 3)), radius=np.zeros(n),
               rect=np.zeros((n, 4), np.int32), valid=np.zeros(n, np.int32))
    ca = camera_array(cam)
    lib.lgso_project(n, _ptr(means), _ptr(quats), _ptr(ls), _ptr(lg), _ptr(ca),
                     _ptr(out["mean2d"]), _ptr(out["depth"]), _ptr(out["conic"]),
                     _ptr(out["opacity"]), _ptr(out["cov2d"]), _ptr(out["radius"]),
                     _ptr(out["rect"]), _ptr(out["valid"]))
    return out


def _crop(cam, crop):
    if crop is None:
        return 0, 0, int(cam.width), int(cam.height)
    return tuple(int(c) for c in crop)


def render(scene, cam, bg=(0.0, 0.0, 0.0), crop=None) -> dict:
    """Brute-force front-to-back compositing of every pixel in ``crop``
    (x0, y0, w, h; default the whole image).  Returns rgb [h,w,3], depth [h,w],
    feat [h,w,D], T_final [h,w], n_contrib [h,w] (int32, number blended),
    margin [h,w] (smallest relative distance of any skip / clamp / stop
    decision of the pixel from its threshold) and zgap [h,w] (smallest
    relative depth gap between consecutive non-skipped Gaussians, which
    decides their order)."""
    lib = _load()
    n = scene.means.shape[0]
    d = scene.feats.shape[1] if scene.feats is not None and scene.feats.ndim == 2 else 0
    x0, y0, w, h = _crop(cam, crop)
    arrs = [_f64(scene.means), _f64(scene.quats), _f64(scene.log_scales),
            _f64(scene.opacity_logits), _f64(scene.colors),
            _f64(scene.feats if d else np.zeros((n, 0)))]
    ca, bga = camera_array(cam), _f64(bg)
    out = dict(rgb=np.zeros((h, w, 3)), depth=np.zeros((h, w)), feat=np.zeros((h, w, d)),
               T_final=np.zeros((h, w)), n_contrib=np.zeros((h, w), np.int32),
               margin=np.zeros((h, w)), zgap=np.zeros((h, w)))
    lib.lgso_render_fwd(n, d, *[_ptr(a) for a in arrs], _ptr(ca), _ptr(bga), x0, y0, w, h,
                        _ptr(out["rgb"]), _ptr(out["depth"]), _ptr(out["feat"]),
                        _ptr(out["T_final"]), _ptr(out["n_contrib"]), _ptr(out["margin"]),
                        _ptr(out["zgap"]))
    return out


def render_backward(scene, cam, g_rgb, g_depth, g_feat, bg=(0.0, 0.0, 0.0), crop=None) -> dict:
    """Analytic backward of :func:`render` for upstream gradients g_* (shaped
    like render's outputs).  Returns gradients w.r.t. means, quats, log_scales,
    opacity_logits, colors, feats and the per-Gaussian 2D gradients ``proj``
    [N,7] = d(u, v, conic a, b, c, opacity, depth)."""
    lib = _load()
    n = scene.means.shape[0]
    d = scene.feats.shape[1] if scene.feats is not None and scene.feats.ndim == 2 else 0
    x0, y0, w, h = _crop(cam, crop)
    arrs = [_f64(scene.means), _f64(scene.quats), _f64(scene.log_scales),
            _f64(scene.opacity_logits), _f64(scene.colors),
            _f64(scene.feats if d else np.zeros((n, 0)))]
    ca, bga = camera_array(cam), _f64(bg)
    gr, gd = _f64(g_rgb).reshape(h, w, 3), _f64(g_depth).reshape(h, w)
    gf = _f64(g_feat if d else np.zeros((h, w, 0))).reshape(h, w, d)
    out = dict(means=np.zeros((n, 3)), quats=np.zeros((n, 4)), log_scales=np.zeros((n, 3)),
               opacity_logits=np.zeros(n), colors=np.zeros((n, 3)), feats=np.zeros((n, d)),
               proj=np.zeros((n, 7)))
    lib.lgso_render_bwd(n, d, *[_ptr(a) for a in arrs], _ptr(ca), _ptr(bga), x0, y0, w, h,
                        _ptr(gr), _ptr(gd), _ptr(gf), _ptr(out["means"]), _ptr(out["quats"]),
                        _ptr(out["log_scales"]), _ptr(out["opacity_logits"]),
                        _ptr(out["colors"]), _ptr(out["feats"]), _ptr(out["proj"]))
    return out


def pose_grad(scene, cam, dproj) -> np.ndarray:
    """Gradient (6,) of the loss w.r.t. a left perturbation exp(xi^) of the
    camera's world->camera transform, xi = (rho, phi), from the per-Gaussian
    2D gradients ``dproj`` [N,7] of this camera (render_backward's ``proj``)."""
    lib = _load()
    n = scene.means.shape[0]
    out = np.zeros(6)
    dp = _f64(dproj)
    lib.lgso_pose_grad(n, _ptr(_f64(scene.means)), _ptr(_f64(scene.quats)),
                       _ptr(_f64(scene.log_scales)), _ptr(_f64(scene.opacity_logits)),
                       _ptr(camera_array(cam)), _ptr(dp), _ptr(out))
    return out


def project_backward(scene, cam, dproj) -> dict:
    """Chain rule from per-Gaussian 2D gradients ``dproj`` [N,7] to the
    parameters of the valid Gaussians."""
    lib = _load()
    n = scene.means.shape[0]
    out = dict(means=np.zeros((n, 3)), quats=np.zeros((n, 4)), log_scales=np.zeros((n, 3)),
               opacity_logits=np.zeros(n))
    arrs = [_f64(scene.means), _f64(scene.quats), _f64(scene.log_scales),
            _f64(scene.opacity_logits)]
    ca, dp = camera_array(cam), _f64(dproj).reshape(n, 7)
    lib.lgso_project_bwd(n, *[_ptr(a) for a in arrs], _ptr(ca), _ptr(dp), _ptr(out["means"]),
                         _ptr(out["quats"]), _ptr(out["log_scales"]),
                         _ptr(out["opacity_logits"]))
    return out


def bin_sort(rect, depth, n, ncams, tiles_x, tiles_y, proj=None) -> dict:
    """Binning definition: emit one key per (camera, Gaussian, reached tile)
    in (camera, index, row-major tile) order, key = ((camera * tiles + tile)
    << 32) | bits(float32 depth); stable sort by key; per-tile ranges.

    ``rect`` int32 [ncams*n, 4] = tile rect [x0, y0, x1, y1); ``depth`` float32
    [ncams*n]; ``proj`` float32 [ncams*n, 8] = the projected records (u, v,
    a, b, c, o, tz, cut): a tile of the rect is reached when the ellipse
    a dx^2 + 2 b dx dy + c dy^2 <= cut meets its pixel-centre square, decided
    in FP32 as the GPU decides it (None: every tile of the rect).  Returns keys
    (uint64 [K]), ids (uint32 [K]) and ranges (uint32 [ncams*tiles, 2])."""
    lib = _load()
    r = np.ascontiguousarray(np.asarray(rect, dtype=np.int32).reshape(-1, 4))
    z = np.ascontiguousarray(np.asarray(depth, dtype=np.float32).reshape(-1))
    pr = None if proj is None else np.ascontiguousarray(
        np.asarray(proj, dtype=np.float32).reshape(-1, 8))
    k = int(lib.lgso_bin_count(n, ncams, _ptr(r), None if pr is None else _ptr(pr)))
    keys = np.zeros(k, np.uint64)
    ids = np.zeros(k, np.uint32)
    ranges = np.zeros((ncams * tiles_x * tiles_y, 2), np.uint32)
    lib.lgso_bin_sort(n, ncams, tiles_x, tiles_y, _ptr(r), _ptr(z),
                      None if pr is None else _ptr(pr), _ptr(keys), _ptr(ids), _ptr(ranges))
    return dict(keys=keys, ids=ids, ranges=ranges)


def l1_loss_grad(pred, target, weight=1.0):
    """Mean absolute error (the L1 terms of Eq. 1) and its gradient, with
    sign(0) = 0; the mean runs over every element of ``pred``."""
    p, t = _f64(pred), _f64(target)
    diff = p - t
    loss = weight * np.abs(diff).mean() if diff.size else 0.0
    return loss, weight * np.sign(diff) / max(diff.size, 1)


def prune_thresholds(min_opacity, max_scale):
    """The geometric thresholds as the float comparisons take them:
    logit(min_opacity) (-inf when min_opacity <= 0) and log(max_scale) (+inf
    when max_scale is not positive and finite), each rounded to float once."""
    import math
    lo = -math.inf if min_opacity <= 0 else math.log(min_opacity / (1.0 - min_opacity))
    hi = math.inf if not (0 < max_scale < math.inf) else math.log(max_scale)
    return float(np.float32(lo)), float(np.float32(hi))


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def prune(means, logits, log_scales, feats, k=8, tau_dist=0.05, tau_sim=0.9,
          min_opacity=0.005, max_scale=float("inf"), idx=None):
    """Language-guided pruning mask (Sec. III-C, Eq. 4) unioned with the
    geometric criteria: uint8 per Gaussian, bit 0 geometric, bit 1 redundant
    (0 keeps the Gaussian).  With ``idx`` only those Gaussians' entries are
    decided (each from scratch) and returned in that order."""
    lib = _load()
    p, lg, ls, f = _f32(means), _f32(logits), _f32(log_scales), _f32(feats)
    n, d = f.shape
    tl, ts = prune_thresholds(min_opacity, max_scale)
    if idx is None:
        out = np.zeros(n, np.uint8)
        rc = lib.lgso_prune(n, d, _ptr(p), _ptr(lg), _ptr(ls), _ptr(f), int(k), float(tau_dist),
                            float(tau_sim), tl, ts, _ptr(out))
    else:
        ix = np.ascontiguousarray(np.asarray(idx, np.int64))
        out = np.zeros(ix.shape[0], np.uint8)
        rc = lib.lgso_prune_sample(n, d, _ptr(p), _ptr(lg), _ptr(ls), _ptr(f), int(k),
                                   float(tau_dist), float(tau_sim), tl, ts, _ptr(ix),
                                   ix.shape[0], _ptr(out))
    if rc != 0:
        raise ValueError("lgso_prune: bad arguments")
    return out
