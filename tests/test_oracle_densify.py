"""Pins of the densification oracle (CPU only): hand-built decisions,
clones exactly duplicated with zero moments for the copy, split samples at
mu + R diag(exp s) z with R from scipy's quaternion rotation and log-scales
reduced by log 1.6, pruning by opacity, and the screen-space statistic of a
single view in closed form."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import densify as D


def small_set():
    rng = np.random.default_rng(1)
    n, P = 6, 14
    p = rng.normal(size=(P, n))
    p[3:6] = np.log([[0.002] * n, [0.004] * n, [0.003] * n])
    p[3:6, 2] = np.log([0.05, 0.02, 0.03])   # large: splits
    p[3:6, 4] = np.log([0.08, 0.01, 0.01])   # large, but pruned
    p[10] = 1.0
    p[10, 4] = -7.0                           # sigma = 0.0009 < 0.005
    m = rng.normal(size=(P, n))
    v = np.abs(rng.normal(size=(P, n)))
    g = np.array([1e-3, 1e-5, 1e-3, 3e-4, 1e-3, 0.0]) * 2
    c = np.array([2, 2, 2, 1, 2, 0], float)   # averages 1e-3, 1e-5, 1e-3, 6e-4, 1e-3, 0
    noise = rng.normal(size=(n, 2, 3))
    return p, m, v, g, c, noise


def test_decisions_clone_split_prune():
    p, m, v, g, c, noise = small_set()
    po, mo, vo, kind = D.densify(p, m, v, g, c, noise, tau=2e-4, dense=0.01, extent=1.0)
    assert list(kind) == [2, 1, 3, 2, 0, 1]
    assert po.shape[1] == 2 + 1 + 2 + 2 + 0 + 1
    # clone of Gaussian 0: identical parameters, moments kept on the first, zero on the copy
    np.testing.assert_array_equal(po[:, 0], p[:, 0])
    np.testing.assert_array_equal(po[:, 1], p[:, 0])
    np.testing.assert_array_equal(mo[:, 0], m[:, 0])
    assert not mo[:, 1].any() and not vo[:, 1].any()
    np.testing.assert_array_equal(po[:, 2], p[:, 1])   # kept unchanged
    np.testing.assert_array_equal(vo[:, 2], v[:, 1])


def test_split_samples_follow_the_covariance():
    p, m, v, g, c, noise = small_set()
    po, mo, vo, kind = D.densify(p, m, v, g, c, noise)
    q = p[6:10, 2]
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()  # scipy: (x, y, z, w), normalises
    s = np.exp(p[3:6, 2])
    for k in range(2):
        out = po[:, 3 + k]
        np.testing.assert_allclose(out[0:3], p[0:3, 2] + R @ (s * noise[2, k]), rtol=0, atol=1e-12)
        np.testing.assert_allclose(out[3:6], p[3:6, 2] - math.log(1.6), rtol=0, atol=1e-12)
        np.testing.assert_array_equal(out[6:], p[6:, 2])
        assert not mo[:, 3 + k].any()
    # the sample covariance of many splits is R diag(s^2) R^T
    rng = np.random.default_rng(7)
    z = rng.normal(size=(200000, 3))
    pts = (R @ (s[:, None] * z.T)).T
    np.testing.assert_allclose(np.cov(pts.T), R @ np.diag(s * s) @ R.T, rtol=0, atol=0.02 * s.max() ** 2)


def test_screen_space_statistic():
    cams = [{"width": 200, "height": 100}, {"width": 64, "height": 64}]
    g2d = [np.array([[0.01, 0.02], [0.0, 0.0]]), np.array([[-0.03, 0.0], [0.5, 0.5]])]
    vis = [np.array([True, True]), np.array([True, False])]
    s, c = D.ndc_grad_stat(g2d, cams, vis)
    assert s[0] == pytest.approx(math.hypot(1.0, 1.0) + math.hypot(0.96, 0.0))
    assert s[1] == 0.0 and list(c) == [2.0, 1.0]
