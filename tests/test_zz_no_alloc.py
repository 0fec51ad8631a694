"""gs_render_bwd_static: the render backward for callers that cannot allocate
device memory (a real-time mapping thread that must not take the device-wide
synchronisation of cudaMalloc, or a host that forbids libraries from owning
device memory).  It uses a fixed scratch array inside the library instead of
the caller's grad2d buffer; its gradients must match gs_render_bwd's within
the gradient tolerance of the other parity tests, on two calls in a row (the
array keeps the previous call's contents).  This file is collected last."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2511_16144_gb300 import synth
from tests.gpu_util import grad_close

pytestmark = pytest.mark.gpu

NAMES = ("means", "quats", "log_scales", "opacity_logits", "colors", "feats")


def test_static_scratch_backward_matches_allocating_call():
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    from paper_2511_16144_gb300 import build, lgs
    from paper_2511_16144_gb300.render import DeviceScene, Frame, zero_grads
    build.build()
    lib = lgs.load()
    cap = int(lib.gs_render_bwd_static_capacity())
    assert cap == 1 << 19

    scene, cams = synth.small_window(n=500, size=32, n_cams=2)
    bg = (0.1, 0.2, 0.3)
    fr = Frame(DeviceScene.from_host(scene), cams, bg)
    gen = torch.Generator(device="cuda").manual_seed(11)
    up = [torch.randn(fr.out[k].shape, device="cuda", generator=gen)
          for k in ("rgb", "depth", "feat")]
    ref = {k: v.cpu().numpy() for k, v in fr.backward(*up).items()}
    assert np.abs(ref["means"]).max() > 0

    for call in range(2):
        grads = zero_grads(fr.scene)
        lgs.gs_render_bwd_static(fr.scene.params(), fr.proj, fr.bufs, fr.cams, fr.scene.colors,
                                 fr.scene.feats, fr.out, *up, grads, bg)
        torch.cuda.synchronize()
        for k in NAMES:
            grad_close(grads[k].cpu().numpy(), ref[k], name=f"call {call}: {k}")

    # sizes beyond the fixed scratch are rejected on the host
    too_many = cap // 2 + 1
    with pytest.raises(lgs.LgsError, match="static scratch"):
        lib_st = lib.gs_render_bwd_static(None, None, None, None, None, None, None, too_many,
                                          lgs.cameras(cams), 2, None, None, 16, 0,
                                          (ctypes.c_float * 3)(0, 0, 0), None, None,
                                          None, None, None, None, None, None, None, None, None,
                                          None)
        lgs._check(lib_st, "gs_render_bwd_static")
