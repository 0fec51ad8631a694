"""GPU parity of language-guided pruning (Sec. III-C, Eq. 4 with the
geometric criteria) and of the compaction that follows it, against the
oracle, bit-exact, through the C ABI (marked gpu)."""
import math

import numpy as np
import pytest
import torch

from paper_2511_16144_gb300 import synth
from tests.gpu_util import bf16_round

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lgs():
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    from paper_2511_16144_gb300 import build, lgs as L
    build.build()
    L.load()
    return L


def _clustered(n, seed, box=1.0, n_blobs=40, blob=0.03, n_feat=6, feat_noise=0.15):
    """Gaussian blobs of points (the surface clusters of a map) with 16-d
    features drawn around a few centroids, opacity logits rounded to 0.1 (so
    ties occur) and log-scales spread across the scale threshold."""
    rng = np.random.default_rng(seed)
    centres = rng.random((n_blobs, 3)) * box
    p = centres[rng.integers(0, n_blobs, n)] + blob * rng.standard_normal((n, 3))
    cent = rng.standard_normal((n_feat, 16))
    f = cent[rng.integers(0, n_feat, n)] + feat_noise * rng.standard_normal((n, 16))
    lg = np.round(rng.standard_normal(n) * 2.0, 1)
    ls = math.log(0.01) + 0.7 * rng.standard_normal((n, 3))
    return (p.astype(np.float32), lg.astype(np.float32), ls.astype(np.float32),
            f.astype(np.float32))


def _run(lgs, p, lg, ls, f, dtype=torch.float32, lo=None, hi=None, **kw):
    lo = p.min(0) if lo is None else lo
    hi = p.max(0) if hi is None else hi
    params = lgs.prune_params(lo, hi, **kw)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    mask, cnt = lgs.gs_prune(t(p), t(lg), t(ls), t(f).to(dtype).contiguous(), params)
    torch.cuda.synchronize()
    assert lgs.lgs_device_error() == 0
    return mask.cpu().numpy(), int(cnt.item())


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("kw", [dict(k=8, tau_dist=0.02, tau_sim=0.9),
                                dict(k=1, tau_dist=0.02, tau_sim=0.9),
                                dict(k=16, tau_dist=0.035, tau_sim=0.7, min_opacity=0.05,
                                     max_scale=0.03)])
def test_prune_matches_oracle(lgs, oracle_lib, dtype, kw):
    p, lg, ls, f = _clustered(6000, 11)
    m, cnt = _run(lgs, p, lg, ls, f, dtype, **kw)
    fo = bf16_round(f) if dtype == torch.bfloat16 else f
    ref = oracle_lib.prune(p, lg, ls, fo, **kw)
    np.testing.assert_array_equal(m, ref)
    assert cnt == int((ref != 0).sum())
    assert (ref & 2).sum() > 100  # the rule fires


@pytest.mark.parametrize("dtype,d,k,tau", [(torch.bfloat16, 12, 8, 0.03),
                                            (torch.float32, 12, 5, 0.035),
                                            (torch.float32, 13, 12, 0.035),
                                            (torch.bfloat16, 64, 16, 0.03)])
def test_prune_feature_widths(lgs, oracle_lib, dtype, d, k, tau):
    """Feature rows read element by element (BF16 widths that are not a
    multiple of 8, FP32 widths not a multiple of 4) or as 16-byte vectors,
    with candidate lists of 8 and 16 entries, on grids of more (0.03) and
    fewer (0.035) than 8 cells per Gaussian."""
    p, lg, ls, f = _clustered(5000, 13)
    rng = np.random.default_rng(14)
    f = np.ascontiguousarray(f[:, rng.integers(0, 16, d)]
                             + 0.05 * rng.standard_normal((5000, d)).astype(np.float32))
    kw = dict(k=k, tau_dist=tau, tau_sim=0.8)
    m, cnt = _run(lgs, p, lg, ls, f, dtype, **kw)
    fo = bf16_round(f) if dtype == torch.bfloat16 else f
    ref = oracle_lib.prune(p, lg, ls, fo, **kw)
    np.testing.assert_array_equal(m, ref)
    assert cnt == int((ref != 0).sum())
    assert (ref & 2).sum() > 100


def test_prune_points_outside_the_bounds(lgs, oracle_lib):
    """Bounds that cover only part of the scene: the border cells absorb the
    rest and the result is unchanged."""
    p, lg, ls, f = _clustered(4000, 12)
    kw = dict(k=8, tau_dist=0.02, tau_sim=0.85)
    ref = oracle_lib.prune(p, lg, ls, f, **kw)
    lo, hi = p.min(0), p.max(0)
    mid = (lo + hi) / 2
    for b in ((lo, hi), (mid - 0.1, mid + 0.1), (mid, mid)):
        m, _ = _run(lgs, p, lg, ls, f, lo=b[0], hi=b[1], **kw)
        np.testing.assert_array_equal(m, ref)


def test_prune_degenerate_inputs(lgs, oracle_lib):
    kw = dict(k=4, tau_dist=0.05, tau_sim=0.5, min_opacity=0.0)
    # every Gaussian at one point with one feature: squared distances all 0,
    # ranking by index, equal logits -> only the first survives
    n = 37
    p = np.zeros((n, 3), np.float32)
    f = np.tile(np.eye(16, dtype=np.float32)[0], (n, 1))
    lg = np.zeros(n, np.float32)
    ls = np.full((n, 3), math.log(0.01), np.float32)
    m, cnt = _run(lgs, p, lg, ls, f, lo=(-1, -1, -1), hi=(1, 1, 1), **kw)
    ref = oracle_lib.prune(p, lg, ls, f, **kw)
    np.testing.assert_array_equal(m, ref)
    assert m[0] == 0 and cnt == int((ref != 0).sum())
    # one Gaussian; zero features
    m, cnt = _run(lgs, p[:1], lg[:1], ls[:1], f[:1], lo=(-1, -1, -1), hi=(1, 1, 1), **kw)
    assert list(m) == [0] and cnt == 0
    f0 = np.zeros((5, 16), np.float32)
    m, _ = _run(lgs, p[:5], lg[:5], ls[:5], f0, lo=(-1, -1, -1), hi=(1, 1, 1), **kw)
    assert list(m) == [0] * 5
    # no Gaussians
    params = lgs.prune_params((0, 0, 0), (1, 1, 1))
    e = torch.empty((0, 3), device="cuda")
    mask, cnt = lgs.gs_prune(e, torch.empty(0, device="cuda"), e, torch.empty((0, 16), device="cuda"),
                             params)
    assert int(cnt.item()) == 0 and mask.numel() == 0


def test_prune_full_size_indoor(lgs, oracle_lib):
    """300k Gaussians in the 6x6x3 m room with spatially coherent 16-d
    features (64 semantic cells): sampled decisions against the oracle, each
    decided from scratch over all Gaussians, and the count."""
    scene, _ = synth.indoor()
    f = synth.semantic_features(scene.means, synth.ROOM_LO, synth.ROOM_HI, dim=16, noise=0.05)
    kw = dict(k=8, tau_dist=0.06, tau_sim=0.9, min_opacity=0.02, max_scale=0.1)
    m, cnt = _run(lgs, scene.means, scene.opacity_logits, scene.log_scales, f,
                  torch.bfloat16, lo=synth.ROOM_LO, hi=synth.ROOM_HI, **kw)
    fo = bf16_round(f)
    rng = np.random.default_rng(5)
    idx = np.concatenate([rng.integers(0, scene.n, 300),
                          rng.choice(np.flatnonzero(m & 2), 150, replace=False)])
    ref = oracle_lib.prune(scene.means, scene.opacity_logits, scene.log_scales, fo, idx=idx, **kw)
    np.testing.assert_array_equal(m[idx], ref)
    assert cnt == int((m != 0).sum())
    assert 0.02 < ((m & 2) != 0).mean() < 0.9


def test_compaction_keeps_rows_in_order(lgs):
    rng = np.random.default_rng(9)
    n = 100_000 + 77
    mask = (rng.random(n) < 0.37).astype(np.uint8) * rng.integers(1, 4, n).astype(np.uint8)
    arrays = [rng.standard_normal((n, 3)).astype(np.float32),
              rng.standard_normal((n, 4)).astype(np.float32),
              rng.integers(0, 2 ** 16, (n, 16)).astype(np.int16),
              rng.standard_normal(n).astype(np.float32),
              rng.integers(0, 2 ** 16, (n, 3)).astype(np.uint16).view(np.int16)]
    t = [torch.from_numpy(a).cuda() for a in arrays]
    out, new_index = lgs.gs_compact(torch.from_numpy(mask).cuda(), t)
    keep = mask == 0
    for a, o in zip(arrays, out):
        np.testing.assert_array_equal(o.cpu().numpy(), a[keep])
    ni = new_index.cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(ni[keep], np.arange(keep.sum()))
    assert (ni[~keep] == 0xFFFFFFFF).all()
    # nothing kept / everything kept
    for mm in (np.ones(n, np.uint8), np.zeros(n, np.uint8)):
        out, _ = lgs.gs_compact(torch.from_numpy(mm).cuda(), t[:1])
        np.testing.assert_array_equal(out[0].cpu().numpy(), arrays[0][mm == 0])
