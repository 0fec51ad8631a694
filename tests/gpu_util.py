"""Helpers shared by the GPU parity tests (host side only)."""
import numpy as np
import torch

from paper_2511_16144_gb300 import synth


def bf16_round(a):
    """float32 array rounded through bfloat16 (what a BF16 channel stores)."""
    return torch.as_tensor(np.asarray(a, np.float32)).bfloat16().float().numpy()


def bf16_scene(scene):
    return synth.Scene(scene.means, scene.quats, scene.log_scales, scene.opacity_logits,
                       bf16_round(scene.colors), bf16_round(scene.feats))


def robust_mask(o, thresh=1e-4, zthresh=1e-6):
    """Pixels whose every skip / clamp / stop decision is farther than
    ``thresh`` (relative) from its threshold in the FP64 oracle, and whose
    consecutive Gaussians differ in depth by more than ``zthresh``
    (relative; FP32 depth resolves about 1.2e-7)."""
    return (o["margin"] > thresh) & (o["zgap"] > zthresh)


def grad_close(g, ref, rel=1e-3, name=""):
    """Per tensor ||g - ref|| <= rel ||ref||, and elementwise |g - ref| <=
    rel * max(|ref|, 1e-2 max|ref|) except for a tiny fraction of entries."""
    g = np.asarray(g, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    nr = np.linalg.norm(ref)
    err = np.linalg.norm(g - ref)
    assert err <= rel * max(nr, 1e-30), f"{name}: |g-ref|={err:.3e} vs {rel}*|ref|={rel * nr:.3e}"
    floor = 1e-2 * np.abs(ref).max() if ref.size else 0.0
    bad = np.abs(g - ref) > rel * np.maximum(np.abs(ref), floor)
    assert bad.mean() <= 1e-3, f"{name}: {bad.sum()} of {bad.size} entries off"
    return err / max(nr, 1e-30)
