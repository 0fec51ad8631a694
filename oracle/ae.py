"""FP64 oracle of the scene-adaptive autoencoder (TEST INFRASTRUCTURE ONLY).

LEGO-SLAM Sec. IV-A.2: encoder E_phi and decoder D_theta are stacks of 1x1
convolutions, i.e. the same MLP applied to every pixel, pretrained as an
autoencoder; Sec. III-B.3 Eq. 2 distils the rendered 16-d map through D_theta
with an L1 loss; Sec. III-B.4 Eq. 3 adapts E_phi alone with an L1 loss against
the rendered map.  The paper fixes neither widths, activation, reduction nor
optimiser; the readings used here:

* widths 512-256-128-64-16 and the mirrored decoder, bias on every layer;
* GELU in its tanh form (Hendrycks & Gimpel, 2016),
  0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))), after every hidden layer,
  linear latent and output (it differs from x Phi(x) by at most 4.7e-4);
* reconstruction loss per pixel = mean_k (y_k - x_k)^2 + (1 - cos(y, x)),
  averaged over the batch; L1 losses are means over all elements;
* Adam, beta = (0.9, 0.999), eps = 1e-8, no weight decay.

A layer is (W [out, in], b [out]) and computes x @ W.T + b.
"""
from __future__ import annotations

import math

import numpy as np

ENC_WIDTHS = (512, 256, 128, 64, 16)
DEC_WIDTHS = (16, 64, 128, 256, 512)


GELU_K = math.sqrt(2.0 / math.pi)
GELU_C = 0.044715


def gelu(x):
    """0.5 x (1 + tanh(u)), u = sqrt(2/pi) (x + 0.044715 x^3)."""
    x = np.asarray(x, np.float64)
    return 0.5 * x * (1.0 + np.tanh(GELU_K * (x + GELU_C * x ** 3)))


def gelu_grad(x):
    """Derivative of :func:`gelu`: 0.5 (1 + t) + 0.5 x (1 - t^2) u'(x)."""
    x = np.asarray(x, np.float64)
    t = np.tanh(GELU_K * (x + GELU_C * x ** 3))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * GELU_K * (1.0 + 3.0 * GELU_C * x * x)


def mlp_forward(layers, x):
    """Runs one MLP (GELU after all but the last layer).  Returns the output
    and the cache [(input, pre-activation)] per layer for the backward."""
    h = np.asarray(x, dtype=np.float64)
    cache = []
    for i, (W, b) in enumerate(layers):
        pre = h @ np.asarray(W, np.float64).T + np.asarray(b, np.float64)
        cache.append((h, pre))
        h = gelu(pre) if i < len(layers) - 1 else pre
    return h, cache


def mlp_backward(layers, cache, dy):
    """Backward of :func:`mlp_forward`: returns dX and [(dW, db)] per layer."""
    grads = [None] * len(layers)
    g = np.asarray(dy, dtype=np.float64)
    for i in range(len(layers) - 1, -1, -1):
        W, _ = layers[i]
        h_in, pre = cache[i]
        if i < len(layers) - 1:
            g = g * gelu_grad(pre)
        grads[i] = (g.T @ h_in, g.sum(axis=0))
        g = g @ np.asarray(W, np.float64)
    return g, grads


def recon_loss(y, x):
    """Per pixel mean_k (y-x)^2 + (1 - cos(y, x)), averaged over pixels;
    returns (loss, dL/dy)."""
    y = np.asarray(y, np.float64)
    x = np.asarray(x, np.float64)
    p, k = y.shape
    diff = y - x
    ny = np.linalg.norm(y, axis=1, keepdims=True)
    nx = np.linalg.norm(x, axis=1, keepdims=True)
    cos = (y * x).sum(axis=1, keepdims=True) / (ny * nx)
    loss = ((diff ** 2).mean(axis=1, keepdims=True) + 1.0 - cos).mean()
    dy = 2.0 * diff / k - (x / (ny * nx) - cos * y / (ny * ny))
    return float(loss), dy / p


def l1_loss(y, t):
    """Mean |y - t| over all elements and its gradient (sign(0) = 0)."""
    d = np.asarray(y, np.float64) - np.asarray(t, np.float64)
    return float(np.abs(d).mean()), np.sign(d) / d.size


def encode(enc, x):
    """z = E_phi(x)."""
    return mlp_forward(enc, x)[0]


def decode(dec, z):
    """y = D_theta(z)."""
    return mlp_forward(dec, z)[0]


def distill(dec, f_render, f_gt):
    """Eq. 2: L_feat = L1(D_theta(F_render), F_gt); returns (loss, dF_render)
    with D_theta frozen."""
    y, cache = mlp_forward(dec, f_render)
    loss, dy = l1_loss(y, f_gt)
    dz, _ = mlp_backward(dec, cache, dy)
    return loss, dz


def adam_update(param, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update in place (step counts from 1)."""
    m *= b1
    m += (1 - b1) * grad
    v *= b2
    v += (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    param -= lr * mh / (np.sqrt(vh) + eps)


def train_step(enc, dec, state, x, target, mode, lr):
    """One optimiser step.

    mode "recon": pretraining as an autoencoder, loss = recon_loss(D(E(x)), x),
    both networks updated.  mode "enc_adapt": Eq. 3, loss = L1(E(x), target)
    with target = F_render, only the encoder updated.

    ``enc``/``dec`` are lists of [W, b] float64 arrays updated in place;
    ``state`` = dict(step=int, m=[...], v=[...]) over enc + dec parameters in
    order (W0, b0, W1, b1, ...).  Returns (loss, grads) with grads taken before
    the update, as [(dW, db)] for enc + dec (None for frozen layers)."""
    z, cache_e = mlp_forward(enc, x)
    if mode == "recon":
        y, cache_d = mlp_forward(dec, z)
        loss, dy = recon_loss(y, x)
        dz, g_dec = mlp_backward(dec, cache_d, dy)
        _, g_enc = mlp_backward(enc, cache_e, dz)
    elif mode == "enc_adapt":
        loss, dz = l1_loss(z, target)
        _, g_enc = mlp_backward(enc, cache_e, dz)
        g_dec = [None] * len(dec)
    else:
        raise ValueError(mode)
    state["step"] += 1
    params = list(enc) + list(dec)
    grads = list(g_enc) + list(g_dec)
    for li, (pw, g) in enumerate(zip(params, grads)):
        if g is None:
            continue
        for j in range(2):
            adam_update(pw[j], g[j], state["m"][2 * li + j], state["v"][2 * li + j],
                        state["step"], lr)
    return loss, grads


def new_state(enc, dec):
    """Zero Adam moments for enc + dec."""
    ms, vs = [], []
    for W, b in list(enc) + list(dec):
        ms += [np.zeros_like(W, np.float64), np.zeros_like(b, np.float64)]
        vs += [np.zeros_like(W, np.float64), np.zeros_like(b, np.float64)]
    return dict(step=0, m=ms, v=vs)


def cosine_error(y, ref, eps=1e-6):
    """Mean over pixels with |ref| > eps of 1 - cos(y, ref); returns
    (mean, number of pixels excluded)."""
    y = np.asarray(y, np.float64)
    ref = np.asarray(ref, np.float64)
    nr = np.linalg.norm(ref, axis=-1)
    ny = np.linalg.norm(y, axis=-1)
    keep = nr > eps
    cos = (y * ref).sum(-1)[keep] / np.maximum(ny[keep] * nr[keep], 1e-300)
    return float((1.0 - cos).mean()) if keep.any() else 0.0, int((~keep).sum())
