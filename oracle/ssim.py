"""FP64 SSIM, PSNR and the D-SSIM training loss (plain numpy).

TEST INFRASTRUCTURE: only the tests and the benchmark's CPU legs use this
module; the product path never does.

The paper evaluates its renders by PSNR and SSIM (Results, Tables II-III);
the 3D-GS training it builds on adds a D-SSIM term to the L1 loss.  The
formulation written out here (the paper fixes none of it):

  window   w = g g^T, g_k = exp(-(k - 5)^2 / (2 1.5^2)) / sum_j (...), k = 0..10
  blur     E[f]_p = sum_q w_(q - p + 5) f_q over the image, f = 0 outside it
           (zero padding; the weights are not renormalised at the borders)
  SSIM map s_p = (2 mx my + C1)(2 sxy + C2) / ((mx^2 + my^2 + C1)(sxx + syy + C2))
           with mx = E[x], my = E[y], sxx = E[x^2] - mx^2, syy = E[y^2] - my^2,
           sxy = E[xy] - mx my, C1 = 0.01^2, C2 = 0.03^2 (data range 1)
  SSIM     mean of s over pixels and channels
  PSNR     10 log10(1 / mean((x - y)^2))
  loss     (1 - lam) mean |x - y| + lam (1 - SSIM), lam = 0.2

The gradient of sum_p s_p with respect to x follows from s_p's partial
derivatives A_p, B_p, C_p with respect to mx, E[x^2] and E[xy] (the blur is
linear and its window symmetric): dS/dx_q = E[A]_q + 2 x_q E[B]_q + y_q E[C]_q.
"""
from __future__ import annotations

import numpy as np

C1 = 0.01 ** 2
C2 = 0.03 ** 2
WIN = 11
SIGMA = 1.5


def window1d(size=WIN, sigma=SIGMA):
    k = np.arange(size, dtype=np.float64) - size // 2
    g = np.exp(-k * k / (2.0 * sigma * sigma))
    return g / g.sum()


def blur(img):
    """Zero-padded separable correlation of the last two axes with the window."""
    g = window1d()
    r = WIN // 2
    img = np.asarray(img, np.float64)
    H, W = img.shape[-2:]
    pad = [(0, 0)] * (img.ndim - 2) + [(r, r), (r, r)]
    p = np.pad(img, pad)
    h = np.zeros(p.shape[:-1] + (W,))
    for k in range(WIN):
        h += g[k] * p[..., :, k:k + W]
    out = np.zeros(img.shape)
    for k in range(WIN):
        out += g[k] * h[..., k:k + H, :]
    return out


def _stats(x, y):
    mx, my = blur(x), blur(y)
    sxx = blur(x * x) - mx * mx
    syy = blur(y * y) - my * my
    sxy = blur(x * y) - mx * my
    n1, n2 = 2.0 * mx * my + C1, 2.0 * sxy + C2
    d1, d2 = mx * mx + my * my + C1, sxx + syy + C2
    return mx, my, n1, n2, d1, d2


def ssim_map(x, y):
    _, _, n1, n2, d1, d2 = _stats(x, y)
    return (n1 * n2) / (d1 * d2)


def ssim(x, y):
    return float(ssim_map(x, y).mean())


def ssim_sum_grad(x, y):
    """d(sum of the SSIM map)/dx."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    mx, my, n1, n2, d1, d2 = _stats(x, y)
    D = d1 * d2
    s = n1 * n2 / D
    A = (2.0 * my * n2 - 2.0 * my * n1) / D - s * (2.0 * mx * d2 - 2.0 * mx * d1) / D
    B = -s / d2
    C = 2.0 * n1 / D
    return blur(A) + 2.0 * x * blur(B) + y * blur(C)


def psnr(x, y):
    d = np.asarray(x, np.float64) - np.asarray(y, np.float64)
    return float(10.0 * np.log10(1.0 / np.mean(d * d)))


def dssim_loss(views_x, views_y, lam=0.2):
    """Loss over a batch of [3, H, W] views: (1 - lam) mean|x - y| + lam (1 -
    SSIM), both means over every (view, channel, pixel); and its gradient per
    view."""
    count = sum(np.asarray(x).size for x in views_x)
    l1 = sum(np.abs(np.asarray(x, np.float64) - np.asarray(y, np.float64)).sum() for x, y in zip(views_x, views_y))
    s = sum(ssim_map(x, y).sum() for x, y in zip(views_x, views_y))
    loss = (1.0 - lam) * l1 / count + lam * (1.0 - s / count)
    grads = []
    for x, y in zip(views_x, views_y):
        d = np.asarray(x, np.float64) - np.asarray(y, np.float64)
        grads.append((1.0 - lam) * np.sign(d) / count - lam * ssim_sum_grad(x, y) / count)
    return float(loss), grads
