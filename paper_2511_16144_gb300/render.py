"""Host-side glue over the C ABI: a device-resident Gaussian map, the
project -> bin -> composite forward, and a torch.autograd.Function whose
backward is gs_render_bwd (LEGO-SLAM Sec. III-B.3: the map is optimised by
gradients of Eq. 1 through the renderer).

Nothing here computes: every step is a liblgs call on the current stream.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import lgs


@dataclass
class DeviceScene:
    """Gaussian parameters on the GPU (structure of arrays)."""
    means: torch.Tensor           # [N,3] f32
    quats: torch.Tensor           # [N,4] f32
    log_scales: torch.Tensor      # [N,3] f32
    opacity_logits: torch.Tensor  # [N]   f32
    colors: torch.Tensor          # [N,3] f32 or bf16
    feats: torch.Tensor           # [N,D] f32 or bf16

    @property
    def n(self):
        return int(self.means.shape[0])

    @staticmethod
    def from_host(scene, device="cuda", chan_dtype=torch.float32):
        t = lambda a, dt=torch.float32: torch.as_tensor(a).to(device=device, dtype=dt).contiguous()
        return DeviceScene(t(scene.means), t(scene.quats), t(scene.log_scales),
                           t(scene.opacity_logits), t(scene.colors, chan_dtype),
                           t(scene.feats, chan_dtype))

    def params(self):
        return (self.means, self.quats, self.log_scales, self.opacity_logits)


class Frame:
    """One forward of a keyframe window: projection, bins and rendered maps,
    kept for the backward."""

    def __init__(self, scene: DeviceScene, cams, bg=(0.0, 0.0, 0.0), bufs=None,
                 want_count=False, want_keys=False, capacity=None):
        self.scene, self.cams, self.bg = scene, list(cams), tuple(float(b) for b in bg)
        tx, ty = lgs.tile_grid(self.cams[0])
        self.proj, self.rect = lgs.gs_project(*scene.params(), self.cams)
        if bufs is None:
            cap = capacity if capacity is not None else max(1 << 16, 16 * scene.n * len(self.cams))
            bufs = lgs.BinBuffers(scene.n, len(self.cams), tx, ty, cap, scene.means.device,
                                  want_keys=want_keys)
        self.bufs = bufs
        self.k = lgs.bin_sort_checked(self.proj, self.rect, bufs)
        self.out = lgs.gs_render_fwd(self.proj, bufs, self.cams, scene.colors, scene.feats,
                                     self.bg, want_count=want_count)

    def backward(self, d_rgb, d_depth, d_feat, grads=None):
        s = self.scene
        if grads is None:
            grads = zero_grads(s)
        grad2d = torch.empty((len(self.cams) * s.n, lgs.PROJ_STRIDE), dtype=torch.float32,
                             device=s.means.device)
        lgs.gs_render_bwd(s.params(), self.proj, self.bufs, self.cams, s.colors, s.feats, self.out,
                          d_rgb.contiguous(), d_depth.contiguous(), d_feat.contiguous(), grads,
                          grad2d, self.bg)
        self.grad2d = grad2d
        return grads


def zero_grads(s: DeviceScene):
    z = lambda t: torch.zeros(t.shape, dtype=torch.float32, device=t.device)
    return dict(means=z(s.means), quats=z(s.quats), log_scales=z(s.log_scales),
                opacity_logits=z(s.opacity_logits), colors=z(s.colors), feats=z(s.feats))


class RenderFunction(torch.autograd.Function):
    """(means, quats, log_scales, opacity_logits, colors, feats) -> (rgb,
    depth, feat) for a fixed keyframe window; backward = gs_render_bwd."""

    @staticmethod
    def forward(ctx, means, quats, log_scales, opacity_logits, colors, feats, cams, bg):
        scene = DeviceScene(means.detach().contiguous(), quats.detach().contiguous(),
                            log_scales.detach().contiguous(), opacity_logits.detach().contiguous(),
                            colors.detach().contiguous(), feats.detach().contiguous())
        fr = Frame(scene, cams, bg)
        ctx.frame = fr
        ctx.chan_dtype = colors.dtype
        return fr.out["rgb"], fr.out["depth"], fr.out["feat"]

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_feat):
        fr = ctx.frame
        g = fr.backward(g_rgb.float(), g_depth.float(), g_feat.float())
        del ctx.frame
        cd = ctx.chan_dtype
        return (g["means"], g["quats"], g["log_scales"], g["opacity_logits"],
                g["colors"].to(cd), g["feats"].to(cd), None, None)


def render(scene: DeviceScene, cams, bg=(0.0, 0.0, 0.0)):
    """Differentiable render of a keyframe window: (rgb, depth, feat)."""
    return RenderFunction.apply(scene.means, scene.quats, scene.log_scales, scene.opacity_logits,
                                scene.colors, scene.feats, list(cams), tuple(bg))
