"""Pins of the point-cloud initialisation oracle (CPU only): crossings of a
sampled sphere field against an independent count of sign changes and the
sphere itself, normals against the radial direction, k-d-tree scales
against brute force, and the rotation taking +z onto the normal."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import init as O


def sphere_volume(n=17, r=0.6):
    ax = np.linspace(-1.0, 1.0, n)
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    return np.sqrt(x * x + y * y + z * z).astype(np.float32), ax[1] - ax[0]


def test_sphere_crossings_count_position_and_normals():
    vol, h = sphere_volume()
    iso = 0.6
    pts, nrm = O.iso_crossings(vol, iso, (-1.0, -1.0, -1.0), (h, h, h))
    inside = vol >= np.float32(iso)
    changes = sum(int((inside[tuple(slice(0, -1) if a == ax else slice(None) for a in range(3))]
                       != inside[tuple(slice(1, None) if a == ax else slice(None) for a in range(3))]).sum())
                  for ax in range(3))
    assert pts.shape[0] == changes > 100
    rad = np.linalg.norm(pts, axis=1)
    assert np.abs(rad - iso).max() <= h * h  # linear interpolation of |x| along an edge
    cosang = np.sum(nrm * pts / rad[:, None], axis=1)
    assert cosang.min() > 0.97  # outward: the field grows with the radius
    np.testing.assert_allclose(np.linalg.norm(nrm, axis=1), 1.0, atol=1e-12)


def test_crossing_order_is_vertex_major_x_fastest():
    vol = np.zeros((3, 3, 4), np.float32)
    vol[1, 1, 2] = 1.0  # one vertex inside: its 6 edges cross
    pts, _ = O.iso_crossings(vol, 0.5, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    # vertices in (z, y, x) order: (2,1,0) +z; (2,0,1) +y; (1,1,1) +x; then (2,1,1): +x, +y, +z
    expect = [(2, 1, 0.5), (2, 0.5, 1), (1.5, 1, 1), (2.5, 1, 1), (2, 1.5, 1), (2, 1, 1.5)]
    np.testing.assert_allclose(pts, expect)


def test_knn_scales_match_brute_force():
    rng = np.random.default_rng(1)
    p = rng.uniform(-1, 1, size=(300, 3)).astype(np.float32)
    p[7] = p[8]  # a duplicate point: distance 0
    np.testing.assert_allclose(O.knn_log_scales(p), O.knn_log_scales_brute(p), rtol=1e-12, atol=1e-12)


def test_init_rotation_takes_z_to_the_normal():
    rng = np.random.default_rng(2)
    nr = rng.normal(size=(50, 3))
    nr /= np.linalg.norm(nr, axis=1, keepdims=True)
    nr[0] = [0.0, 0.0, -1.0]
    p = rng.uniform(size=(50, 3))
    out = O.init_gaussians(p, nr)
    q = out[6:10].T  # (w, x, y, z)
    R = Rotation.from_quat(np.stack([q[:, 1], q[:, 2], q[:, 3], q[:, 0]], axis=1)).as_matrix()
    np.testing.assert_allclose(R[:, :, 2], nr, atol=1e-12)
    assert out[5, 0] == pytest.approx(out[3, 0] + math.log(0.3))
    c = 0.1 + 0.9 * max(0.0, float(nr[3] @ np.ones(3)) / math.sqrt(3))
    assert 0.5 + out[11, 3] / (2 * math.sqrt(math.pi)) == pytest.approx(c)
