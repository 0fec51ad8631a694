"""Render forward and backward at other feature widths (the feature-dimension
ablation of Sec. IV: d = 8 ... 128 channels) against the oracle (marked gpu)."""
import numpy as np
import pytest
import torch

from paper_2511_16144_gb300 import synth
from tests.gpu_util import bf16_scene, grad_close, robust_mask
from tests.test_gpu_render import _check_maps, _frame, _gpu_grads, _np, _upstream

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lgs():
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    from paper_2511_16144_gb300 import build, lgs as L
    build.build()
    L.load()
    return L


@pytest.mark.parametrize("d,chan", [(8, "f32"), (8, "bf16"), (24, "f32"), (32, "bf16"),
                                    (64, "f32"), (128, "bf16")])
def test_render_feature_width(lgs, oracle_lib, d, chan):
    scene, cams = synth.tiny()
    rng = np.random.default_rng(100 + d)
    scene = scene.with_feats(synth.unit_rows(rng.standard_normal((scene.n, d))).astype(np.float32))
    tch = torch.float32 if chan == "f32" else torch.bfloat16
    bg = (0.1, 0.2, 0.3)
    fr = _frame(scene, cams, bg, chan=tch)
    ref = scene if chan == "f32" else bf16_scene(scene)
    o = oracle_lib.render(ref, cams[0], bg=bg)
    out = {k: _np(v[0]) for k, v in fr.out.items() if v is not None}
    assert out["feat"].shape[-1] == d
    _check_maps(out, o, robust_mask(o))
    keep = robust_mask(o, 1e-3)
    g = _upstream(o["depth"].shape, d, keep, 40 + d)
    gg = _gpu_grads(fr, g)
    go = oracle_lib.render_backward(ref, cams[0], *g, bg=bg)
    for k in ("colors", "feats", "opacity_logits", "means", "log_scales", "quats"):
        grad_close(gg[k], go[k], name=k)
