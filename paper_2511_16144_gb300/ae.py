"""Device-resident autoencoder parameters and optimiser state, marshalled
into the lgs_ae_weights / lgs_ae_state structs of the C ABI.

The scene-adaptive encoder E_phi and decoder D_theta (LEGO-SLAM Sec. IV-A.2,
Eq. 2, Eq. 3) are an 8-layer per-pixel MLP 512-256-128-64-16-64-128-256-512;
all arithmetic runs in liblgs (ae_encode, ae_decode, ae_train_step).
"""
from __future__ import annotations

import torch

from . import lgs


class AutoEncoder:
    """FP32 master weights, Adam moments, gradients and BF16 copies on the
    GPU.  ``enc``/``dec`` are lists of (W [out, in], b [out]) host arrays."""

    def __init__(self, enc, dec, device="cuda"):
        layers = list(enc) + list(dec)
        assert len(layers) == lgs.AE_LAYERS
        f = lambda a: torch.as_tensor(a).to(device=device, dtype=torch.float32).contiguous()
        self.W = [f(W) for W, _ in layers]
        self.b = [f(b) for _, b in layers]
        for l, W in enumerate(self.W):
            assert tuple(W.shape) == (lgs.AE_WIDTHS[l + 1], lgs.AE_WIDTHS[l]), (l, W.shape)
        z = lambda t: torch.zeros_like(t)
        self.mW, self.vW = [z(W) for W in self.W], [z(W) for W in self.W]
        self.mb, self.vb = [z(b) for b in self.b], [z(b) for b in self.b]
        # gradients as consecutive views of one buffer (gW_0, gb_0, gW_1, ...):
        # the training step zeroes them with a single memset
        flat = torch.zeros(sum(W.numel() + b.numel() for W, b in zip(self.W, self.b)),
                           dtype=torch.float32, device=device)
        self.gW, self.gb, o = [], [], 0
        for W, b in zip(self.W, self.b):
            self.gW.append(flat[o:o + W.numel()].view(W.shape))
            o += W.numel()
            self.gb.append(flat[o:o + b.numel()].view(b.shape))
            o += b.numel()
        self.Wbf = [torch.empty(W.shape, dtype=torch.bfloat16, device=device) for W in self.W]
        self.Wtbf = [torch.empty((W.shape[1], W.shape[0]), dtype=torch.bfloat16, device=device)
                     for W in self.W]
        self.state = lgs.AeState()
        for name in ("W", "b", "mW", "vW", "mb", "vb", "gW", "gb", "Wbf", "Wtbf"):
            arr = getattr(self.state, name)
            for l, t in enumerate(getattr(self, name)):
                arr[l] = t.data_ptr()
        self.state.step = 0
        self.weights = lgs.AeWeights()
        for l in range(lgs.AE_LAYERS):
            self.weights.W[l] = self.Wbf[l].data_ptr()
            self.weights.Wt[l] = self.Wtbf[l].data_ptr()
            self.weights.b[l] = self.b[l].data_ptr()
        self._ws = {}
        lgs.ae_pack(self.state)

    @property
    def step(self):
        return int(self.state.step)

    def _cached(self, key, ws):
        self._ws[key] = ws
        return ws

    def encode(self, x):
        """z [P,16] f32 from x bf16 [P,512]."""
        z = torch.empty((x.shape[0], 16), dtype=torch.float32, device=x.device)
        self._cached("enc", lgs.ae_encode(self.weights, x, z, self._ws.get("enc")))
        return z

    def decode(self, z):
        """y [P,512] f32 = D(z)."""
        y = torch.empty((z.shape[0], 512), dtype=torch.float32, device=z.device)
        self._cached("dec", lgs.ae_decode(self.weights, z, y=y, ws=self._ws.get("dec")))
        return y

    def distill(self, z, target, weight=1.0, loss=None):
        """Eq. 2 through the frozen decoder: returns (loss [1], dz [P,16])."""
        loss = torch.zeros(1, device=z.device) if loss is None else loss
        dz = torch.empty_like(z)
        self._cached("dec", lgs.ae_decode(self.weights, z, target, weight, loss, dz,
                                          ws=self._ws.get("dec")))
        return loss, dz

    def train_step(self, x, target=None, mode=lgs.AE_RECON, lr=1e-3, loss=None):
        loss = torch.zeros(1, device=x.device) if loss is None else loss
        self._cached("train", lgs.ae_train_step(self.state, x, target, mode, lr, loss,
                                                self._ws.get("train")))
        return loss

    def host_layers(self):
        """(enc, dec) as float64 numpy lists of [W, b] (master weights)."""
        L = [[W.double().cpu().numpy(), b.double().cpu().numpy()] for W, b in zip(self.W, self.b)]
        return L[:4], L[4:]
