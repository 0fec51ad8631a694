"""Device-side error reporting through lgs_sync_status (marked gpu).

Every error here is made on the host: non-finite values written into the
Gaussian parameters, an instance buffer one short of what the frame needs,
and a polling limit of one round for the look-back of the sort behind
gs_prune (lgs_set_sort_wait_limit), so that a look-back which finds a slower
block still unpublished gives up.  No wait is left without a bound and no
access leaves its buffer: the calls return, the status comes back through
lgs_sync_status, and the next call on the same context gives the usual
results.
"""
import math

import numpy as np
import pytest
import torch

from paper_2511_16144_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lgs():
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    from paper_2511_16144_gb300 import build, lgs as L
    build.build()
    L.load()
    # errors are recorded per device and process-wide: drop what earlier
    # tests left pending (an overflow test leaves LGS_ERR_CAPACITY behind)
    for _ in range(8):
        if L.lgs_sync_status()[0] == L.OK:
            break
    assert L.lgs_sync_status() == (L.OK, 0)
    return L


def _np(t):
    return t.detach().cpu().numpy()


def test_nonfinite_gaussians_are_culled_and_reported(lgs):
    from paper_2511_16144_gb300.render import DeviceScene
    scene, cams = synth.tiny()
    ds = DeviceScene.from_host(scene)
    clean_p, clean_r = lgs.gs_project(*ds.params(), cams)
    assert lgs.lgs_sync_status() == (lgs.OK, 0)
    bad = {"means": (41, 1, float("nan")), "opacity_logits": (17, None, float("inf")),
           "quats": (1500, 3, float("-inf")), "log_scales": (900, 0, float("nan"))}
    params = [t.clone() for t in ds.params()]
    names = ("means", "quats", "log_scales", "opacity_logits")
    for k, (i, j, v) in bad.items():
        t = params[names.index(k)]
        if j is None:
            t[i] = v
        else:
            t[i, j] = v
    cams2 = [cams[0], synth.Camera(110.0, 110.0, 60.0, 40.0, 128, 96, cams[0].viewmat)]
    proj, rect = lgs.gs_project(*params, cams2)
    st, detail = lgs.lgs_sync_status()
    assert st == lgs.ERR_NONFINITE and detail == 17, (st, detail)
    assert lgs.lgs_sync_status() == (lgs.OK, 0)  # reported once
    n = scene.n
    idx = np.array(sorted(i for i, _, _ in bad.values()))
    p, r = _np(proj).reshape(2, n, 8), _np(rect).reshape(2, n, 4)
    assert np.all(p[:, idx] == 0) and np.all(r[:, idx] == 0)
    keep = np.setdiff1d(np.arange(n), idx)
    np.testing.assert_array_equal(p[0, keep], _np(clean_p)[keep])
    np.testing.assert_array_equal(r[0, keep], _np(clean_r)[keep])
    # a NaN in a camera is refused before anything is enqueued
    badcam = synth.Camera(float("nan"), 110.0, 60.0, 40.0, 128, 96, cams[0].viewmat)
    with pytest.raises(lgs.LgsError) as e:
        lgs.gs_project(*ds.params(), [cams[0], badcam])
    assert e.value.status == lgs.ERR_NONFINITE


def test_capacity_overflow_is_reported_with_the_required_count(lgs):
    from paper_2511_16144_gb300.render import DeviceScene
    scene, cams = synth.tiny()
    ds = DeviceScene.from_host(scene)
    proj, rect = lgs.gs_project(*ds.params(), cams)
    tx, ty = lgs.tile_grid(cams[0])
    big = lgs.BinBuffers(scene.n, 1, tx, ty, 1 << 18, "cuda")
    lgs.gs_bin_sort(proj, rect, big)
    assert lgs.lgs_sync_status() == (lgs.OK, 0)
    k = int(big.k_dev.item())
    small = lgs.BinBuffers(scene.n, 1, tx, ty, k - 1, "cuda")
    lgs.gs_bin_sort(proj, rect, small)
    # a NaN Gaussian in the same window: both are pending, non-finite first
    bad = ds.means.clone()
    bad[3, 0] = float("nan")
    lgs.gs_project(bad, ds.quats, ds.log_scales, ds.opacity_logits, cams)
    assert lgs.lgs_sync_status() == (lgs.ERR_NONFINITE, 3)
    assert lgs.lgs_sync_status() == (lgs.ERR_CAPACITY, k)
    assert lgs.lgs_sync_status() == (lgs.OK, 0)
    assert int(_np(small.ranges).sum()) == 0
    # the mapping step's own check raises with the count it needs
    from paper_2511_16144_gb300.pipeline import MappingStep
    (rgb_t, dep_t, f_t), = synth.targets(cams, feat_dim=16)
    step = MappingStep(ds, cams, torch.from_numpy(rgb_t[None]).cuda(),
                       torch.from_numpy(dep_t[None]).cuda(),
                       torch.from_numpy(f_t.reshape(-1, 16)).cuda().bfloat16(), capacity=k - 1)
    step.run()
    with pytest.raises(lgs.LgsError) as e:
        step.check()
    assert e.value.status == lgs.ERR_CAPACITY and e.value.detail == k


def _prune_inputs(n, seed):
    rng = np.random.default_rng(seed)
    means = torch.from_numpy((rng.random((n, 3)) * 8.0).astype(np.float32)).cuda()
    logits = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).cuda()
    ls = torch.from_numpy((math.log(0.02) + 0.5 * rng.standard_normal((n, 3))).astype(np.float32)).cuda()
    feats = torch.from_numpy(rng.standard_normal((n, 8)).astype(np.float32)).cuda().bfloat16()
    return means, logits, ls, feats


def test_sort_wait_timeout_is_reported(lgs):
    """With a one-round polling limit some look-back of the cell sort finds
    an earlier block still unpublished and gives up; the call returns, the
    timeout comes back with the sort's wait-site bits, and with the default
    limit the same call gives the same mask as before."""
    n = 1 << 22
    means, logits, ls, feats = _prune_inputs(n, 21)
    params = lgs.prune_params((0, 0, 0), (8, 8, 8), k=4, tau_dist=0.05, tau_sim=0.5)
    ws = torch.empty(int(lgs.load().gs_prune_workspace(n)), dtype=torch.uint8, device="cuda")
    mask0, cnt0 = lgs.gs_prune(means, logits, ls, feats, params, ws=ws)
    assert lgs.lgs_sync_status() == (lgs.OK, 0)
    mask0 = mask0.clone()
    seen = None
    try:
        lgs.lgs_set_sort_wait_limit(1)
        for attempt in range(20):
            lgs.gs_prune(means, logits, ls, feats, params, ws=ws)
            st, detail = lgs.lgs_sync_status()
            assert st in (lgs.OK, lgs.ERR_TIMEOUT), st
            if st == lgs.ERR_TIMEOUT:
                seen = (attempt, detail)
                break
    finally:
        lgs.lgs_set_sort_wait_limit(0)
    print(f"timeout after {seen}")
    assert seen is not None, "no look-back had to wait in 20 calls"
    assert seen[1] & (0xF << 8) and not seen[1] & ~(0xF << 8), hex(seen[1])
    assert lgs.lgs_sync_status() == (lgs.OK, 0)
    assert lgs.lgs_device_error() == 0
    mask1, cnt1 = lgs.gs_prune(means, logits, ls, feats, params, ws=ws)
    assert lgs.lgs_sync_status() == (lgs.OK, 0)
    assert torch.equal(mask1, mask0) and int(cnt1.item()) == int(cnt0.item())
