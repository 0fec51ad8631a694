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


def decided_target(dec_rounded, z_rounded, rng, delta=0.05):
    """An F_gt for the gradient of Eq. 2 whose every sign(y - F_gt) is
    decided with room to spare: F_gt = y* - s delta, with y* the oracle's
    decoder output for z and s a random sign, rounded to BF16.  The L1
    gradient is a sign, so wherever |y - F_gt| is below the rounding of the
    BF16 activations (about 4e-3 |y|) the GPU and the oracle may take
    opposite signs at a tie; with this target every difference is near
    delta, and dz compares the arithmetic alone."""
    from oracle import ae
    y = ae.decode(dec_rounded, z_rounded)
    s = rng.choice(np.array([-1.0, 1.0]), size=y.shape)
    return bf16_round(y - s * delta)
