"""FP64 oracle of the D-SSIM term of the photometric loss (TEST INFRASTRUCTURE
ONLY: only tests/, the smoke check and the CPU legs of the benchmark use it).

LEGO-SLAM Sec. III-B.3 (Eq. 1): L_rgb combines an L1 term and a D-SSIM term
between the rendered and the observed image.  The paper gives neither the
weights nor the SSIM parameters; the readings here are the ones of the
standard 3DGS photometric loss:

* SSIM (Wang et al., 2004) per colour channel with an 11 x 11 Gaussian window
  of standard deviation 1.5 (normalised to sum 1), images zero-padded at the
  border ("same" filtering), C1 = 0.01^2, C2 = 0.03^2 (unit data range):
  SSIM = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_x^2 + s_y^2 + C2))
  with mu = G * x, s_x^2 = G * x^2 - mu_x^2, s_xy = G * xy - mu_x mu_y;
* D-SSIM = 1 - mean SSIM over all pixels and channels;
* L_rgb = (1 - lambda) L1 + lambda D-SSIM with lambda = 0.2.

Images are [..., H, W, 3] float arrays (pixels in rows, channels last).
"""
from __future__ import annotations

import numpy as np
from scipy.signal import convolve2d

WINDOW = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2
LAMBDA = 0.2


def window_1d(size=WINDOW, sigma=SIGMA):
    """Normalised 1D Gaussian taps; the 2D window is their outer product."""
    x = np.arange(size, dtype=np.float64) - (size - 1) / 2.0
    g = np.exp(-x * x / (2.0 * sigma * sigma))
    return g / g.sum()


def _blur(img):
    """'same' 2D filtering of one [H, W] map with the Gaussian window, zero
    outside the image (the window is symmetric, so filtering = convolution)."""
    g = window_1d()
    return convolve2d(img, np.outer(g, g), mode="same", boundary="fill", fillvalue=0.0)


def ssim_map(x, y):
    """Per-pixel, per-channel SSIM of x against y ([..., H, W, 3])."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    out = np.empty(np.broadcast_shapes(x.shape, y.shape))
    for idx in np.ndindex(*x.shape[:-3], x.shape[-1]):
        lead, ch = idx[:-1], idx[-1]
        xi = x[lead + (slice(None), slice(None), ch)]
        yi = y[lead + (slice(None), slice(None), ch)]
        mx, my = _blur(xi), _blur(yi)
        sxx = _blur(xi * xi) - mx * mx
        syy = _blur(yi * yi) - my * my
        sxy = _blur(xi * yi) - mx * my
        out[lead + (slice(None), slice(None), ch)] = (
            (2 * mx * my + C1) * (2 * sxy + C2) / ((mx * mx + my * my + C1) * (sxx + syy + C2)))
    return out


def dssim_loss(x, y, weight=1.0):
    """weight * (1 - mean SSIM(x, y)) and its gradient with respect to x.

    With s = dL/dSSIM at each pixel: dL/dmu_x = s dSSIM/dmu_x, b = dL/ds_x^2,
    c = dL/ds_xy; because mu_x, s_x^2 and s_xy are window sums of x, x^2 and
    xy, dL/dx = G * (dL/dmu_x - 2 mu_x b - mu_y c) + 2 x (G * b) + y (G * c)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    n = x.size
    s = -weight / n
    grad = np.empty_like(x)
    total = 0.0
    for idx in np.ndindex(*x.shape[:-3], x.shape[-1]):
        lead, ch = idx[:-1], idx[-1]
        sl = lead + (slice(None), slice(None), ch)
        xi, yi = x[sl], y[sl]
        mx, my = _blur(xi), _blur(yi)
        sxx = _blur(xi * xi) - mx * mx
        syy = _blur(yi * yi) - my * my
        sxy = _blur(xi * yi) - mx * my
        a1, a2 = 2 * mx * my + C1, 2 * sxy + C2
        b1, b2 = mx * mx + my * my + C1, sxx + syy + C2
        ssim = a1 * a2 / (b1 * b2)
        total += ssim.sum()
        d_mx = s * (2 * my * a2 / (b1 * b2) - 2 * mx * ssim / b1)
        b = -s * ssim / b2
        c = s * 2 * a1 / (b1 * b2)
        a = d_mx - 2 * mx * b - my * c
        grad[sl] = _blur(a) + 2 * xi * _blur(b) + yi * _blur(c)
    return float(weight * (1.0 - total / n)), grad


def rgb_loss(x, y, lam=LAMBDA, weight=1.0):
    """weight * ((1 - lam) mean|x - y| + lam D-SSIM(x, y)) and its gradient."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    d = x - y
    l1 = np.abs(d).mean()
    g1 = np.sign(d) / d.size
    ld, gd = dssim_loss(x, y)
    return (float(weight * ((1 - lam) * l1 + lam * ld)),
            weight * ((1 - lam) * g1 + lam * gd))
