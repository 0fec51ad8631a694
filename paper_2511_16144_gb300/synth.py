"""Seeded synthetic inputs shared by the CUDA path's tests, the benchmark and
the CPU oracle.

This module only draws data: Gaussian scenes, camera poses, target images,
512-d embedding maps and autoencoder initial weights.  It holds none of the
method's arithmetic (no projection, compositing, loss or network code), so
both sides can take their inputs from it without sharing any computation.
Everything is float32 numpy; the caller moves it to the device.

Workloads (scene seed = 1000 + index, target seed = 2000 + index, autoencoder
seed = 3000 + index):

* ``tiny``      128x96, fx=fy=120, 2,000 Gaussians in [-1,1]^2 x [1,3] in
                front of an identity camera, 8 feature clusters.
* ``indoor``    640x480, fx=fy=525, c=(320,240), 300k Gaussians uniform in a
                6x6x3 m room, 32 clusters; keyframes on a 2 m-radius arc.
* ``outdoor``   1200x680, fx=fy=600, 2M Gaussians in 40x40x8 m,
                log-scales ~ N(ln 0.08, 0.6), 64 clusters, 10 m-radius arc.
* ``embedding`` per-frame 640x480 maps of 512-d unit embeddings, piecewise
                constant over 64 Voronoi cells plus N(0, 0.02) noise.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

ZNEAR = 0.2


@dataclass
class Camera:
    """Pinhole camera; ``viewmat`` is the row-major 3x4 world-to-camera
    transform [R | t] in OpenCV axes (x right, y down, z forward)."""
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    viewmat: np.ndarray
    znear: float = ZNEAR


@dataclass
class Scene:
    """Structure-of-arrays Gaussian parameters (float32)."""
    means: np.ndarray           # [N, 3]
    quats: np.ndarray           # [N, 4] (w, x, y, z), not necessarily unit
    log_scales: np.ndarray      # [N, 3]
    opacity_logits: np.ndarray  # [N]
    colors: np.ndarray          # [N, 3]
    feats: np.ndarray           # [N, D]

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        return Scene(*(np.ascontiguousarray(a[idx]) for a in
                       (self.means, self.quats, self.log_scales, self.opacity_logits,
                        self.colors, self.feats)))

    def with_feats(self, feats) -> "Scene":
        return Scene(self.means, self.quats, self.log_scales, self.opacity_logits, self.colors,
                     np.ascontiguousarray(feats, dtype=np.float32))


def unit_rows(x: np.ndarray) -> np.ndarray:
    """Rows scaled to unit length (data preparation of the embeddings)."""
    return x / np.linalg.norm(x, axis=-1, keepdims=True)


def clustered_features(rng, n, dim, n_clusters, noise):
    """n unit vectors: a random one of ``n_clusters`` unit centroids plus
    N(0, noise^2) per component, renormalised."""
    cent = unit_rows(rng.standard_normal((n_clusters, dim)))
    k = rng.integers(0, n_clusters, size=n)
    return unit_rows(cent[k] + noise * rng.standard_normal((n, dim))).astype(np.float32)


def random_scene(rng, n, lo, hi, log_scale_mean, log_scale_std, n_clusters, feat_dim=16,
                 feat_noise=0.05) -> Scene:
    """Gaussians uniform in the box [lo, hi]; log-scales ~ N(mean, std) per
    axis; quaternions uniform on S^3; opacity logits ~ N(0, 1); RGB ~ U[0,1];
    clustered unit features."""
    lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
    means = (lo + (hi - lo) * rng.random((n, 3))).astype(np.float32)
    log_scales = (log_scale_mean + log_scale_std * rng.standard_normal((n, 3))).astype(np.float32)
    quats = unit_rows(rng.standard_normal((n, 4))).astype(np.float32)
    logits = rng.standard_normal(n).astype(np.float32)
    colors = rng.random((n, 3)).astype(np.float32)
    feats = clustered_features(rng, n, feat_dim, n_clusters, feat_noise)
    return Scene(means, quats, log_scales, logits, colors, feats)


def look_at(eye, target, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """World-to-camera [R | t] (3x4) of a camera at ``eye`` looking at
    ``target``: rows of R are (right, down, forward)."""
    eye, target, up = (np.asarray(v, np.float64) for v in (eye, target, up))
    fwd = target - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])
    return np.concatenate([R, (-R @ eye)[:, None]], axis=1).astype(np.float32)


def arc_cameras(n, center, radius, height, f, width, height_px, cx, cy, arc=math.pi / 2):
    """``n`` cameras evenly over an ``arc`` (radians, ends included) of a
    circle of ``radius`` at z = ``height`` around ``center``, each looking at
    ``center``."""
    cams = []
    for k in range(n):
        th = arc * k / max(n - 1, 1)
        eye = (center[0] + radius * math.cos(th), center[1] + radius * math.sin(th), height)
        cams.append(Camera(f, f, cx, cy, width, height_px, look_at(eye, center)))
    return cams


def identity_view() -> np.ndarray:
    return np.concatenate([np.eye(3), np.zeros((3, 1))], axis=1).astype(np.float32)


# --------------------------------------------------------------------------
# workloads

def tiny(seed: int = 1000):
    """128x96 frame, 2,000 Gaussians, 8 clusters, identity camera."""
    rng = np.random.default_rng(seed)
    scene = random_scene(rng, 2000, (-1, -1, 1), (1, 1, 3), math.log(0.03), 0.4, 8)
    cam = Camera(120.0, 120.0, 64.0, 48.0, 128, 96, identity_view())
    return scene, [cam]


ROOM_LO, ROOM_HI = (0.0, 0.0, 0.0), (6.0, 6.0, 3.0)
ROOM_CENTER = (3.0, 3.0, 1.5)


def indoor(n: int = 300_000, n_cams: int = 1, seed: int = 1001):
    """640x480 keyframes (fx=fy=525, c=(320,240)) on a 2 m arc at 1.5 m height
    around the room centre; 300k Gaussians uniform in the 6x6x3 m room with
    32 feature clusters.  ``n_cams`` = 1 gives the first keyframe alone."""
    rng = np.random.default_rng(seed)
    scene = random_scene(rng, n, ROOM_LO, ROOM_HI, math.log(0.03), 0.4, 32)
    cams = arc_cameras(8, ROOM_CENTER, 2.0, 1.5, 525.0, 640, 480, 320.0, 240.0)
    return scene, cams[:n_cams]


def outdoor(n: int = 2_000_000, n_cams: int = 8, seed: int = 1004):
    """1200x680 keyframes (fx=fy=600, c=(600,340)) on a 10 m arc at 2 m height
    around the centre of a 40x40x8 m volume; log-scales ~ N(ln 0.08, 0.6),
    64 clusters."""
    rng = np.random.default_rng(seed)
    scene = random_scene(rng, n, (0, 0, 0), (40, 40, 8), math.log(0.08), 0.6, 64)
    cams = arc_cameras(8, (20.0, 20.0, 4.0), 10.0, 2.0, 600.0, 1200, 680, 600.0, 340.0)
    return scene, cams[:n_cams]


def small_window(n: int = 500, size: int = 32, n_cams: int = 1, seed: int = 1002):
    """Finite-difference sub-scene: ``n`` Gaussians in [-0.6,0.6]^2 x [1.5,2.5]
    seen by ``size`` x ``size`` cameras (fx=fy=30) near the identity pose;
    log-scales ~ N(ln 0.06, 0.3) so splats cover a few pixels."""
    rng = np.random.default_rng(seed)
    scene = random_scene(rng, n, (-0.6, -0.6, 1.5), (0.6, 0.6, 2.5), math.log(0.06), 0.3, 8)
    cams = []
    for k in range(n_cams):
        eye = (0.1 * k, -0.05 * k, 0.0)
        cams.append(Camera(30.0, 30.0, size / 2, size / 2, size, size,
                           look_at(eye, (0.1 * k, -0.05 * k, 2.0), up=(0.0, -1.0, 0.0))))
    return scene, cams


def targets(cams, feat_dim=16, seed: int = 2000):
    """Seeded per-camera targets: RGB ~ U[0,1], depth ~ U[0.5, 5], unit
    features of ``feat_dim`` (HWC, float32)."""
    rng = np.random.default_rng(seed)
    out = []
    for c in cams:
        h, w = c.height, c.width
        rgb = rng.random((h, w, 3)).astype(np.float32)
        dep = (0.5 + 4.5 * rng.random((h, w))).astype(np.float32)
        feat = unit_rows(rng.standard_normal((h, w, feat_dim))).astype(np.float32)
        out.append((rgb, dep, feat))
    return out


def embedding_centroids(n: int = 64, dim: int = 512, seed: int = 1003):
    """Scene-fixed unit 512-d centroids of the embedding maps."""
    return unit_rows(np.random.default_rng(seed).standard_normal((n, dim))).astype(np.float32)


def embedding_map(rng, centroids, width=640, height=480, n_seeds=64, noise=0.02):
    """One frame of 512-d embeddings: ``n_seeds`` Voronoi seeds uniform in the
    image (nearest seed, ties to the lower index), each cell taking a random
    scene centroid, plus N(0, noise^2), renormalised.  [H, W, 512] float32."""
    seeds = rng.random((n_seeds, 2)) * (width, height)
    cell_cent = rng.integers(0, centroids.shape[0], size=n_seeds)
    ys, xs = np.mgrid[0:height, 0:width]
    px = np.stack([xs + 0.5, ys + 0.5], -1).reshape(-1, 2)
    best = np.zeros(px.shape[0], np.int64)
    bestd = np.full(px.shape[0], np.inf)
    for s in range(n_seeds):
        dd = ((px - seeds[s]) ** 2).sum(-1)
        upd = dd < bestd
        best[upd] = s
        bestd[upd] = dd[upd]
    base = centroids[cell_cent[best]]
    emb = unit_rows(base + noise * rng.standard_normal(base.shape).astype(np.float32))
    return emb.reshape(height, width, -1).astype(np.float32)


def embedding_scene(n: int = 100_000, seed: int = 1003, dim: int = 512):
    """Indoor-room Gaussians whose ``feats`` are 512-d: a random scene
    centroid plus N(0, 0.02^2), renormalised (the plain 512-channel path)."""
    rng = np.random.default_rng(seed + 10)
    scene = random_scene(rng, n, ROOM_LO, ROOM_HI, math.log(0.03), 0.4, 8)
    cent = embedding_centroids(dim=dim, seed=seed)
    k = rng.integers(0, cent.shape[0], size=n)
    g = unit_rows(cent[k] + 0.02 * rng.standard_normal((n, dim)).astype(np.float32))
    cams = arc_cameras(8, ROOM_CENTER, 2.0, 1.5, 525.0, 640, 480, 320.0, 240.0)
    return scene.with_feats(g.astype(np.float32)), cams


def semantic_features(means, lo, hi, n_cells=64, dim=512, noise=0.02, seed=1005):
    """Spatially coherent 512-d semantics: ``n_cells`` Voronoi seeds uniform in
    the box [lo, hi], each cell owning one unit centroid; a Gaussian takes its
    nearest seed's centroid plus N(0, noise^2), renormalised (the 3D analogue
    of the per-frame Voronoi embedding maps).  [N, dim] float32."""
    rng = np.random.default_rng(seed)
    lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
    seeds = lo + (hi - lo) * rng.random((n_cells, 3))
    cent = unit_rows(rng.standard_normal((n_cells, dim)))
    m = np.asarray(means, np.float64)
    best = np.zeros(m.shape[0], np.int64)
    bestd = np.full(m.shape[0], np.inf)
    for k in range(n_cells):
        d = ((m - seeds[k]) ** 2).sum(-1)
        upd = d < bestd
        best[upd] = k
        bestd[upd] = d[upd]
    g = cent[best] + noise * rng.standard_normal((m.shape[0], dim))
    return unit_rows(g).astype(np.float32)


def synthetic_records(rng, rect, depth, opacity_range=(0.01, 1.0)):
    """Projected records (u, v, a, b, c, o, tz, cut) for binning inputs (no
    projection arithmetic): the mean uniform over the rect's pixel span
    widened by 8 px, a random positive-definite conic (principal standard
    deviations 1-40 px at a random angle), opacity uniform in
    ``opacity_range``, depth as given and the tile-test cutoff
    2 ln(255 o) 1.001 + 0.01.  float32 [m, 8]."""
    m = rect.shape[0]
    x0, y0, x1, y1 = (rect[:, k].astype(np.float64) for k in range(4))
    u = 16.0 * x0 - 8.0 + rng.random(m) * (16.0 * np.maximum(x1 - x0, 1) + 16.0)
    v = 16.0 * y0 - 8.0 + rng.random(m) * (16.0 * np.maximum(y1 - y0, 1) + 16.0)
    s1 = np.exp(rng.uniform(np.log(1.0), np.log(40.0), m))
    s2 = np.exp(rng.uniform(np.log(1.0), np.log(40.0), m))
    th = rng.uniform(0.0, np.pi, m)
    ct, st = np.cos(th), np.sin(th)
    # conic = R diag(1/s1^2, 1/s2^2) R^T
    a = ct * ct / s1 ** 2 + st * st / s2 ** 2
    b = ct * st * (1.0 / s1 ** 2 - 1.0 / s2 ** 2)
    c = st * st / s1 ** 2 + ct * ct / s2 ** 2
    o = rng.uniform(*opacity_range, m)
    cut = 2.0 * np.log(255.0 * o) * 1.001 + 0.01
    rec = np.stack([u, v, a, b, c, o, np.asarray(depth, np.float64), cut], -1)
    return rec.astype(np.float32)


def semantic_features_device(means, lo, hi, n_cells=64, dim=512, noise=0.02, seed=1005,
                             out_dtype=None):
    """The recipe of :func:`semantic_features` generated on the device of
    ``means`` (a torch tensor [N, 3]) with torch's seeded generator, for maps
    too large to build on the host (2M Gaussians x 512 channels): seeds and
    centroids as there, nearest seed per Gaussian (ties to the lower index),
    centroid plus N(0, noise^2) noise, renormalised.  The noise stream differs
    from the host version's.  Returns [N, dim] in ``out_dtype`` (default
    float32), built in chunks of 2^18 rows."""
    import torch
    rng = np.random.default_rng(seed)
    lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
    seeds = lo + (hi - lo) * rng.random((n_cells, 3))
    cent = unit_rows(rng.standard_normal((n_cells, dim)))
    dev = means.device
    sd = torch.as_tensor(seeds, dtype=torch.float64, device=dev)
    ct = torch.as_tensor(cent, dtype=torch.float32, device=dev)
    gen = torch.Generator(device=dev).manual_seed(seed)
    n = int(means.shape[0])
    out = torch.empty((n, dim), dtype=out_dtype or torch.float32, device=dev)
    for a in range(0, n, 1 << 18):
        m = means[a:a + (1 << 18)].double()
        d = ((m[:, None, :] - sd[None]) ** 2).sum(-1)           # [rows, n_cells]
        best = torch.argmin(d, dim=1)                            # first minimum
        g = ct[best] + noise * torch.randn((m.shape[0], dim), device=dev, generator=gen)
        out[a:a + m.shape[0]] = (g / g.norm(dim=1, keepdim=True)).to(out.dtype)
    return out


def ae_init(widths_enc=(512, 256, 128, 64, 16), widths_dec=(16, 64, 128, 256, 512),
            seed: int = 3003):
    """Initial autoencoder weights, each layer (W [out, in], b [out]) ~
    U(-1/sqrt(fan_in), 1/sqrt(fan_in)).  Returns (enc, dec) lists."""
    rng = np.random.default_rng(seed)

    def stack(widths):
        out = []
        for a, b in zip(widths[:-1], widths[1:]):
            bound = 1.0 / math.sqrt(a)
            W = rng.uniform(-bound, bound, (b, a)).astype(np.float32)
            bb = rng.uniform(-bound, bound, b).astype(np.float32)
            out.append([W, bb])
        return out

    return stack(widths_enc), stack(widths_dec)


def synthetic_projected(rng, n, ncams, tiles_x, tiles_y, max_extent=6, tie_frac=0.05):
    """Random binning inputs (no projection arithmetic): per (camera,
    Gaussian) a tile rect [x0, y0, x1, y1) inside the grid (about 10% empty)
    and a positive float32 depth, with ``tie_frac`` of the depths copied from
    another Gaussian so equal keys occur.  Returns (rect int32 [ncams*n, 4],
    depth float32 [ncams*n])."""
    m = ncams * n
    x0 = rng.integers(0, tiles_x, m)
    y0 = rng.integers(0, tiles_y, m)
    w = rng.integers(1, max_extent + 1, m)
    h = rng.integers(1, max_extent + 1, m)
    x1 = np.minimum(x0 + w, tiles_x)
    y1 = np.minimum(y0 + h, tiles_y)
    empty = rng.random(m) < 0.1
    x1 = np.where(empty, x0, x1)
    y1 = np.where(empty, y0, y1)
    rect = np.stack([x0, y0, x1, y1], -1).astype(np.int32)
    depth = (0.2 + 10.0 * rng.random(m)).astype(np.float32)
    ties = rng.random(m) < tie_frac
    src = rng.integers(0, m, m)
    depth = np.where(ties, depth[src], depth).astype(np.float32)
    return rect, depth
