"""One mapping-loop step on the GPU, with every buffer preallocated so the
step can be captured in a CUDA graph and replayed.

LEGO-SLAM Sec. III-B.3: each map-optimisation iteration renders a keyframe
and minimises L_total = L_rgb + w_depth L_depth + w_feat L_feat (Eq. 1), with
L_feat = L1(D_theta(F_render), F_gt) through the frozen decoder (Eq. 2).
The step here is: gs_project -> gs_bin_sort -> gs_render_fwd -> L1 terms of
RGB and depth -> ae_decode (decoder, L1 against F_gt, gradient to F_render)
-> gs_render_bwd (raster backward + projection chain rule).  The plain path
renders all 512 feature channels and takes the L1 against F_gt directly.

Only liblgs kernels compute; torch provides the memory.
"""
from __future__ import annotations

import ctypes

import torch

from . import lgs
from .render import DeviceScene, zero_grads


class MappingStep:
    """Buffers and calls of one mapping step for a fixed keyframe window.

    scene: DeviceScene (feats [N,16] for the compressed path, [N,512] for the
    plain path); cams: cameras sharing one image size; rgb_t [C,H,W,3] and
    depth_t [C,H,W] float32 targets; feat_t bf16 [C*H*W, 512] (F_gt);
    model: AutoEncoder (compressed path) or None (plain path)."""

    def __init__(self, scene: DeviceScene, cams, rgb_t, depth_t, feat_t, model=None,
                 w_depth=0.1, w_feat=1.0, bg=(0.0, 0.0, 0.0), capacity=None):
        self.lib = lgs.load()
        self.scene, self.cams = scene, list(cams)
        self.model = model
        self.w_depth, self.w_feat = float(w_depth), float(w_feat)
        self.bg = (ctypes.c_float * 3)(*[float(b) for b in bg])
        self.ca = lgs.cameras(self.cams)
        c, n = len(self.cams), scene.n
        h, w = int(self.cams[0].height), int(self.cams[0].width)
        self.pixels = c * h * w
        self.D = int(scene.feats.shape[1])
        dev = scene.means.device
        self.proj = torch.empty((c * n, lgs.PROJ_STRIDE), dtype=torch.float32, device=dev)
        self.rect = torch.empty((c * n, 4), dtype=torch.int16, device=dev)
        tx, ty = lgs.tile_grid(self.cams[0])
        if capacity is None:
            # size the instance buffer from one eager binning pass
            probe = lgs.BinBuffers(n, c, tx, ty, max(1 << 16, 16 * n * c), dev)
            p, r = lgs.gs_project(*scene.params(), self.cams)
            k = lgs.bin_sort_checked(p, r, probe)
            capacity = int(k * 1.25) + 4096
        self.bufs = lgs.BinBuffers(n, c, tx, ty, capacity, dev)
        f32 = lambda *s: torch.empty(s, dtype=torch.float32, device=dev)
        self.out = dict(rgb=f32(c, h, w, 3), depth=f32(c, h, w), feat=f32(c, h, w, self.D),
                        T_final=f32(c, h, w),
                        last=torch.empty((c, h, w), dtype=torch.int32, device=dev))
        self.rgb_t, self.depth_t, self.feat_t = rgb_t, depth_t, feat_t
        self.d_rgb, self.d_depth, self.d_feat = f32(c, h, w, 3), f32(c, h, w), f32(c, h, w, self.D)
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)
        self.grads = zero_grads(scene)
        self.grad2d = f32(c * n, lgs.PROJ_STRIDE)
        if model is not None:
            assert self.D == 16, "the compressed path renders 16 channels"
            self.ae_ws = torch.empty(max(lgs.ae_workspace_bytes(self.pixels, lgs.AE_DECODE), 256),
                                     dtype=torch.uint8, device=dev)
        else:
            assert self.D == feat_t.shape[-1], "the plain path renders every F_gt channel"
        self.k_dev = self.bufs.k_dev

    def calls(self):
        """The step as an ordered list of (name, enqueue-function) pairs, one
        per C-ABI call group, each enqueueing on the current stream."""
        L, sc, b = self.lib, self.scene, self.bufs
        p, chk = lgs._p, lgs._check
        c = len(self.cams)
        o, g = self.out, self.grads

        def project():
            chk(L.gs_project(p(sc.means), p(sc.quats), p(sc.log_scales), p(sc.opacity_logits),
                             sc.n, self.ca, c, p(self.proj), p(self.rect), lgs._stream()),
                "gs_project")

        def bin_sort():
            chk(L.gs_bin_sort(p(self.proj), p(self.rect), b.n, b.n_cams, b.tiles_x, b.tiles_y,
                              b.capacity, p(b.ids), p(b.ranges), None, p(b.k_dev),
                              p(b.workspace), b.workspace_bytes, lgs._stream()), "gs_bin_sort")

        def render_fwd():
            chk(L.gs_render_fwd(p(self.proj), p(b.ids), p(b.ranges), sc.n, self.ca, c,
                                p(sc.colors), p(sc.feats), self.D, lgs._dtype_code(sc.feats),
                                self.bg, p(o["rgb"]), p(o["depth"]), p(o["feat"]),
                                p(o["T_final"]), p(o["last"]), None, lgs._stream()),
                "gs_render_fwd")

        def zero_loss():
            chk(L.lgs_zero(p(self.loss), 4, lgs._stream()), "lgs_zero")

        def l1_terms():
            s = lgs._stream()
            chk(L.lgs_l1_loss(p(o["rgb"]), p(self.rgb_t), lgs.F32, o["rgb"].numel(), 1.0,
                              p(self.d_rgb), p(self.loss), s), "lgs_l1_loss")
            chk(L.lgs_l1_loss(p(o["depth"]), p(self.depth_t), lgs.F32, o["depth"].numel(),
                              self.w_depth, p(self.d_depth), p(self.loss), s), "lgs_l1_loss")
            if self.model is None:
                chk(L.lgs_l1_loss(p(o["feat"]), p(self.feat_t), lgs.BF16, o["feat"].numel(),
                                  self.w_feat, p(self.d_feat), p(self.loss), s), "lgs_l1_loss")

        def decode():
            chk(L.ae_decode(ctypes.byref(self.model.weights), p(o["feat"]), self.pixels,
                            p(self.feat_t), self.w_feat, p(self.loss), p(self.d_feat), None,
                            p(self.ae_ws), self.ae_ws.numel(), lgs._stream()), "ae_decode")

        def losses():
            zero_loss()
            l1_terms()

        def zero_grads():
            s = lgs._stream()
            for t in g.values():
                chk(L.lgs_zero(p(t), t.numel() * 4, s), "lgs_zero")

        def backward():
            s = lgs._stream()
            chk(L.gs_render_bwd(p(sc.means), p(sc.quats), p(sc.log_scales), p(sc.opacity_logits),
                                p(self.proj), p(b.ids), p(b.ranges), sc.n, self.ca, c,
                                p(sc.colors), p(sc.feats), self.D, lgs._dtype_code(sc.feats),
                                self.bg, p(o["T_final"]), p(o["last"]), p(self.d_rgb),
                                p(self.d_depth), p(self.d_feat), p(self.grad2d), p(g["means"]),
                                p(g["quats"]), p(g["log_scales"]), p(g["opacity_logits"]),
                                p(g["colors"]), p(g["feats"]), s), "gs_render_bwd")

        def render_bwd():
            zero_grads()
            backward()

        self._parts = dict(zero_loss=zero_loss, l1_terms=l1_terms, decode=decode,
                           zero_grads=zero_grads, backward=backward)
        out = [("gs_project", project), ("gs_bin_sort", bin_sort),
               ("gs_render_fwd", render_fwd), ("l1_losses", losses)]
        if self.model is not None:
            out.append(("ae_decode", decode))
        out.append(("gs_render_bwd", render_bwd))
        return out

    def run(self):
        """Enqueues one step on the current stream (no synchronisation).

        With the decoder, the L1 terms of RGB and depth and the zeroing of the
        parameter gradients do not depend on it: they run on a side stream
        beside it (a parallel branch when the step is captured in a graph),
        joined before the backward.  The loss is zeroed before the fork, as
        both branches add to it.  (Packing the decoder weights on the side
        stream from the start of the step, with ae_decode_pack and
        ae_decode_packed, measured 6 us slower: it competes with projection
        and binning for the SMs.)"""
        calls = self.calls()
        if self.model is None:
            for _, fn in calls:
                fn()
            return
        fns = dict(calls)
        part = self._parts
        for name in ("gs_project", "gs_bin_sort", "gs_render_fwd"):
            fns[name]()
        part["zero_loss"]()
        main = torch.cuda.current_stream()
        if getattr(self, "_side", None) is None or self._side.device != main.device:
            self._side = torch.cuda.Stream(device=main.device)
        fork, join = torch.cuda.Event(), torch.cuda.Event()
        fork.record(main)
        self._side.wait_event(fork)
        with torch.cuda.stream(self._side):
            part["l1_terms"]()
            part["zero_grads"]()
            join.record(self._side)
        part["decode"]()
        main.wait_event(join)
        part["backward"]()

    def check(self):
        """Synchronises the current stream and raises LgsError for an error
        the device recorded while running the step: above all
        LGS_ERR_CAPACITY when a frame needs more instances than the bin
        buffer (sized once, from the first frame) holds -- its ranges are
        then empty and the step renders background with zero gradients --
        with the count it needs as ``detail`` (rebuild the step with that
        capacity)."""
        lgs.check_device("mapping step")

    def count_blended(self):
        """Number blended per pixel for the last forward (re-runs the forward
        with the counting output)."""
        L, sc, b, p, o = self.lib, self.scene, self.bufs, lgs._p, self.out
        cnt = torch.empty_like(o["last"])
        lgs._check(L.gs_render_fwd(p(self.proj), p(b.ids), p(b.ranges), sc.n, self.ca,
                                   len(self.cams), p(sc.colors), p(sc.feats), self.D,
                                   lgs._dtype_code(sc.feats), self.bg, p(o["rgb"]), p(o["depth"]),
                                   p(o["feat"]), p(o["T_final"]), p(o["last"]), p(cnt),
                                   lgs._stream()), "gs_render_fwd")
        return cnt
