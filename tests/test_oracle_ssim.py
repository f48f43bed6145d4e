"""Pins of the FP64 SSIM / PSNR / D-SSIM oracle (CPU only): the blur against
scipy's correlation, SSIM of an image with itself, the closed form of
constant images away from the border, PSNR of a constant offset, and the
analytic gradients against central finite differences."""
import math

import numpy as np
import pytest

from oracle import ssim as S


def test_blur_is_scipy_zero_padded_correlation():
    from scipy.ndimage import correlate
    rng = np.random.default_rng(1)
    img = rng.uniform(size=(2, 23, 31))
    g = S.window1d()
    w2 = np.outer(g, g)
    assert abs(g.sum() - 1.0) < 1e-15 and np.argmax(g) == 5 and g[0] == pytest.approx(math.exp(-25 / 4.5) / sum(
        math.exp(-(k - 5) ** 2 / 4.5) for k in range(11)))
    for c in range(2):
        ref = correlate(img[c], w2, mode="constant", cval=0.0)
        np.testing.assert_allclose(S.blur(img)[c], ref, rtol=0, atol=1e-14)


def test_ssim_of_an_image_with_itself_is_one():
    rng = np.random.default_rng(2)
    x = rng.uniform(size=(3, 20, 17))
    np.testing.assert_allclose(S.ssim_map(x, x), 1.0, rtol=0, atol=1e-12)


def test_ssim_of_constant_images_away_from_the_border():
    a, b = 0.3, 0.7
    x = np.full((1, 40, 40), a)
    y = np.full((1, 40, 40), b)
    s = S.ssim_map(x, y)[0, 5:-5, 5:-5]   # the window lies inside the image
    np.testing.assert_allclose(s, (2 * a * b + S.C1) / (a * a + b * b + S.C1), rtol=1e-12)
    # a structure term: x = y + c has sxx = syy = sxy, so only luminance differs
    rng = np.random.default_rng(3)
    y = rng.uniform(0.2, 0.6, size=(1, 30, 30))
    x = y + 0.1
    m = S.ssim_map(x, y)[0, 5:-5, 5:-5]
    mx, my = S.blur(x)[0, 5:-5, 5:-5], S.blur(y)[0, 5:-5, 5:-5]
    np.testing.assert_allclose(m, (2 * mx * my + S.C1) / (mx * mx + my * my + S.C1), rtol=1e-10)


def test_psnr_of_a_constant_offset():
    rng = np.random.default_rng(4)
    y = rng.uniform(size=(3, 12, 9))
    assert S.psnr(y + 0.05, y) == pytest.approx(10 * math.log10(1 / 0.05 ** 2), rel=1e-12)


def test_ssim_gradient_matches_central_differences():
    rng = np.random.default_rng(5)
    x = rng.uniform(size=(2, 14, 13))
    y = np.clip(x + rng.normal(0, 0.1, size=x.shape), 0, 1)
    g = S.ssim_sum_grad(x, y)
    h = 1e-6
    for _ in range(40):
        c, i, j = rng.integers(0, 2), rng.integers(0, 14), rng.integers(0, 13)
        xp, xm = x.copy(), x.copy()
        xp[c, i, j] += h
        xm[c, i, j] -= h
        fd = (S.ssim_map(xp, y).sum() - S.ssim_map(xm, y).sum()) / (2 * h)
        assert g[c, i, j] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_dssim_loss_gradient_matches_central_differences():
    rng = np.random.default_rng(6)
    xs = [rng.uniform(size=(3, 9, 11)), rng.uniform(size=(3, 12, 7))]
    ys = [rng.uniform(size=(3, 9, 11)), rng.uniform(size=(3, 12, 7))]
    loss, grads = S.dssim_loss(xs, ys, 0.2)
    h = 1e-6
    for _ in range(30):
        v = int(rng.integers(0, 2))
        c, i, j = (int(rng.integers(0, n)) for n in xs[v].shape)
        xp = [x.copy() for x in xs]
        xm = [x.copy() for x in xs]
        xp[v][c, i, j] += h
        xm[v][c, i, j] -= h
        fd = (S.dssim_loss(xp, ys, 0.2)[0] - S.dssim_loss(xm, ys, 0.2)[0]) / (2 * h)
        assert grads[v][c, i, j] == pytest.approx(fd, rel=1e-5, abs=1e-9)
