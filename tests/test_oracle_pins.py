"""Pins of the FP64 oracle against closed forms, library routines, invariants
and finite differences (CPU only).

Each test fixes a part of the oracle by something other than the oracle's own
formula: a closed-form image of a special configuration, a library routine
(scipy spherical harmonics / rotations, torch Adam), an invariance of the
mathematics, or central finite differences of the whole render.
"""
import math

import numpy as np
import pytest
import torch

from paper_2509_05216_gb300 import inputs as I

Y00 = 0.5 / math.sqrt(math.pi)


def logit(p):
    return math.log(p / (1.0 - p))


def one_scene(means, log_scales, quats, opac, rgb, deg=0):
    n = len(means)
    k = (deg + 1) ** 2
    sh = np.zeros((n, k, 3))
    sh[:, 0, :] = (np.asarray(rgb, np.float64) - 0.5) / Y00
    return I.pack_params(np.asarray(means, np.float64), np.asarray(log_scales, np.float64),
                         np.asarray(quats, np.float64), np.asarray(opac, np.float64), sh)


def eff(sc):
    """(rgb [n,3], sigma [n]) from the FP32-rounded parameters (degree-0 colour)."""
    P = sc["params"].astype(np.float64)
    n = sc["n"]
    rgb = np.stack([Y00 * P[11 + c, :n] + 0.5 for c in range(3)], axis=1)
    return rgb, 1.0 / (1.0 + np.exp(-P[10, :n]))


def axis_camera(size, distance=3.0, bg=(0.0, 0.0, 0.0)):
    return I.pinhole(I.look_at((0.0, 0.0, distance), up=(0.0, 1.0, 0.0)), size, size, bg=bg)


def closed_form_alpha(cam, s2x, s2y, mux, muy, sig):
    """alpha image of an axis-aligned 2D Gaussian with covariance diag(s2x, s2y)."""
    H, W = cam["height"], cam["width"]
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    G = np.exp(-0.5 * ((x - mux) ** 2 / s2x + (y - muy) ** 2 / s2y))
    return np.minimum(0.99, sig * G), G, x - mux, y - muy


def rect_mask(cam, mux, muy, r):
    """Pixels of the tiles whose index range is [floor((mu-r)/16), floor((mu+r+15)/16))."""
    H, W = cam["height"], cam["width"]
    gw, gh = (W + 15) // 16, (H + 15) // 16
    x0 = min(gw, max(0, math.floor((mux - r) / 16)))
    x1 = min(gw, max(0, math.floor((mux + r + 15) / 16)))
    y0 = min(gh, max(0, math.floor((muy - r) / 16)))
    y1 = min(gh, max(0, math.floor((muy + r + 15) / 16)))
    m = np.zeros((H, W), bool)
    m[16 * y0:16 * y1, 16 * x0:16 * x1] = True
    return m


# ---------------------------------------------------------------- closed forms

def test_single_isotropic_gaussian_image_and_gradient(oracle):
    cam = axis_camera(64)
    d, s, rgb, o = 3.0, math.log(0.05), (0.7, 0.4, 0.55), 0.3
    sc = one_scene([[0, 0, 0]], [[s, s, s]], [[1, 0, 0, 0]], [o], [rgb])
    img, tf, mg, _ = oracle.render(sc, cam)
    # closed form on the FP32-rounded parameters the oracle actually sees
    P = sc["params"].astype(np.float64)
    s, o = P[3, 0], P[10, 0]
    rgb = tuple(Y00 * P[11 + c, 0] + 0.5 for c in range(3))
    fx = cam["fx"]
    s2 = (fx * math.exp(s) / d) ** 2 + 0.3
    sig = 1.0 / (1.0 + math.exp(-o))
    a, G, dx, dy = closed_form_alpha(cam, s2, s2, cam["cx"], cam["cy"], sig)
    r = math.ceil(3.0 * math.sqrt(s2 + math.sqrt(0.1)))
    use = (a >= 1.0 / 255.0) & rect_mask(cam, cam["cx"], cam["cy"], r)
    a = np.where(use, a, 0.0)
    for c in range(3):
        np.testing.assert_allclose(img[c], rgb[c] * a, rtol=0, atol=1e-12)
    np.testing.assert_allclose(tf, 1.0 - a, rtol=0, atol=1e-12)
    assert not mg.any()

    # gradient of L = sum(dimg * image) against the closed-form derivatives
    rng = np.random.default_rng(5)
    dimg = rng.normal(size=img.shape)
    grad = oracle.render_grad(sc, [cam], [dimg])
    w = dimg * use  # only contributing pixels
    wrgb = sum(w[c] * rgb[c] for c in range(3))
    # d/d sh0_c = Y00 * alpha
    for c in range(3):
        assert grad[11 + c, 0] == pytest.approx(Y00 * np.sum(w[c] * a), rel=1e-9, abs=1e-12)
    # d/d o: alpha = sigma(o) G
    assert grad[10, 0] == pytest.approx(np.sum(wrgb * G * sig * (1 - sig)), rel=1e-9)
    # d/d s_x: Sigma'_xx = (fx/d)^2 e^{2 s_x} + 0.3
    ds2 = 2.0 * (fx / d) ** 2 * math.exp(2 * s)
    assert grad[3, 0] == pytest.approx(np.sum(wrgb * a * 0.5 * dx ** 2 / s2 ** 2 * ds2), rel=1e-9)
    assert grad[4, 0] == pytest.approx(np.sum(wrgb * a * 0.5 * dy ** 2 / s2 ** 2 * ds2), rel=1e-9)
    assert abs(grad[5, 0]) < 1e-12          # depth axis: no effect at the image centre
    assert np.all(np.abs(grad[6:10, 0]) < 1e-12)   # isotropic: rotation has no effect
    # d/d mu_x: mu2D_x = fx t_x / t_z + cx with t_x = mu_x (camera x = world x)
    # (dx, dy are pixel minus mean, so d alpha / d mu2D_x = alpha dx / s2)
    assert grad[0, 0] == pytest.approx(np.sum(wrgb * a * dx / s2) * fx / d, rel=1e-9)
    # camera y = -world y
    assert grad[1, 0] == pytest.approx(-np.sum(wrgb * a * dy / s2) * fx / d, rel=1e-9)
    # d/d mu_z: t_z = d - mu_z scales Sigma' by (fx e^s / t_z)^2
    ds2z = (fx * math.exp(s)) ** 2 * 2.0 / d ** 3
    expect = np.sum(wrgb * a * 0.5 * (dx ** 2 + dy ** 2) / s2 ** 2 * ds2z)
    assert grad[2, 0] == pytest.approx(expect, rel=1e-9)


def test_anisotropic_rotated_about_view_axis(oracle):
    """Scales (sx, sy) rotated by theta about the view axis: Sigma' closed form."""
    from scipy.spatial.transform import Rotation
    cam = axis_camera(64)
    d, fx = 3.0, cam["fx"]
    sx, sy, th = 0.08, 0.03, 0.6
    q_xyzw = Rotation.from_euler("z", th).as_quat()
    q = [q_xyzw[3], q_xyzw[0], q_xyzw[1], q_xyzw[2]]
    sc = one_scene([[0, 0, 0]], [[math.log(sx), math.log(sy), math.log(0.01)]], [q], [0.0],
                   [(0.5, 0.5, 0.5)])
    pr = oracle.project(sc, cam)
    P = sc["params"][:, 0].astype(np.float64)     # the FP32-rounded values
    Rz = Rotation.from_quat([P[7], P[8], P[9], P[6]]).as_matrix()
    sx, sy, sz = np.exp(P[3:6])
    Sw = Rz @ np.diag([sx * sx, sy * sy, sz * sz]) @ Rz.T
    Wc = np.diag([1.0, -1.0, -1.0])       # camera axes: x right, y down, z forward
    S2 = (fx / d) ** 2 * (Wc @ Sw @ Wc.T)[:2, :2] + 0.3 * np.eye(2)
    conic = np.linalg.inv(S2)
    np.testing.assert_allclose(pr["conic"][0], [conic[0, 0], conic[0, 1], conic[1, 1]], rtol=1e-12)


def test_two_gaussians_front_to_back(oracle):
    cam = axis_camera(65)  # odd size: the centre pixel is the principal point
    c1, c2 = (0.9, 0.1, 0.2), (0.1, 0.2, 0.9)
    a1, a2 = 0.5, 0.6
    # index 0 is the far one: order must come from depth, not index
    sc = one_scene([[0, 0, 0], [0, 0, 0.5]], [[-3, -3, -3]] * 2, [[1, 0, 0, 0]] * 2,
                   [logit(a2), logit(a1)], [c2, c1])
    img, tf, _, _ = oracle.render(sc, cam)
    (c2, c1), (a2, a1) = eff(sc)
    for c in range(3):
        assert img[c, 32, 32] == pytest.approx(c1[c] * a1 + c2[c] * a2 * (1 - a1), rel=1e-12)
    assert tf[32, 32] == pytest.approx((1 - a1) * (1 - a2), rel=1e-12)


def test_equal_depth_ties_follow_index(oracle):
    cam = axis_camera(65)
    c0, c1 = (0.9, 0.1, 0.2), (0.1, 0.2, 0.9)
    sc = one_scene([[0, 0, 0], [0, 0, 0]], [[-3, -3, -3]] * 2, [[1, 0, 0, 0]] * 2,
                   [logit(0.7), logit(0.4)], [c0, c1])
    img, _, _, _ = oracle.render(sc, cam)
    (c0, c1), (a0, a1) = eff(sc)
    for c in range(3):
        assert img[c, 32, 32] == pytest.approx(c0[c] * a0 + c1[c] * a1 * (1 - a0), rel=1e-12)


def test_transmittance_stop_excludes_the_crossing_gaussian(oracle):
    cam = axis_camera(65)
    n = 20
    rng = np.random.default_rng(3)
    cols = rng.uniform(0.1, 0.9, size=(n, 3))
    zs = np.linspace(0.5, -0.5, n)       # index order == depth order
    sc = one_scene([[0, 0, z] for z in zs], [[-3, -3, -3]] * n, [[1, 0, 0, 0]] * n,
                   [0.0] * n, cols)
    img, tf, _, _ = oracle.render(sc, cam)
    cols, _ = eff(sc)
    # alpha = 0.5 each; 0.5^14 < 1e-4 <= 0.5^13, so 13 Gaussians composite
    k = 13
    expect = sum(cols[j] * 0.5 * 0.5 ** j for j in range(k))
    np.testing.assert_allclose(img[:, 32, 32], expect, rtol=1e-12)
    assert tf[32, 32] == pytest.approx(0.5 ** k, rel=1e-12)


def test_alpha_clamp_and_zero_gradient_through_it(oracle):
    cam = axis_camera(65, bg=(0.2, 0.3, 0.4))
    col = (0.8, 0.6, 0.3)
    sc = one_scene([[0, 0, 0]], [[-3, -3, -3]], [[1, 0, 0, 0]], [10.0], [col])
    img, _, _, _ = oracle.render(sc, cam)
    col = eff(sc)[0][0]
    for c in range(3):
        assert img[c, 32, 32] == pytest.approx(col[c] * 0.99 + 0.01 * cam["bg"][c], rel=1e-12)
    dimg = np.zeros_like(img)
    dimg[:, 32, 32] = 1.0
    g = oracle.render_grad(sc, [cam], [dimg])
    assert g[10, 0] == 0.0                       # opacity: clamped alpha
    assert abs(g[0, 0]) < 1e-12 and abs(g[1, 0]) < 1e-12
    for c in range(3):
        assert g[11 + c, 0] == pytest.approx(Y00 * 0.99, rel=1e-12)


def test_alpha_below_skip_threshold_gives_background(oracle):
    cam = axis_camera(64, bg=(0.1, 0.2, 0.3))
    sc = one_scene([[0, 0, 0]], [[-2, -2, -2]], [[1, 0, 0, 0]], [logit(0.0035)], [(1, 1, 1)])
    img, tf, _, _ = oracle.render(sc, cam)
    for c in range(3):
        assert np.all(img[c] == np.float64(np.float32(cam["bg"][c])))
    assert np.all(tf == 1.0)


def test_tile_rect_decides_membership(oracle):
    """A wide Gaussian still has alpha > 1/255 just left of its rect; the pixel
    there must stay background, the first pixel inside must not."""
    cam = axis_camera(256)
    fx, d = cam["fx"], 3.0
    s2 = 900.0
    s = math.log(d * math.sqrt(s2 - 0.3) / fx)
    col = (0.5, 0.5, 0.5)
    sc = one_scene([[0, 0, 0]], [[s, s, s]], [[1, 0, 0, 0]], [logit(0.99)], [col])
    img, _, _, _ = oracle.render(sc, cam)
    P = sc["params"].astype(np.float64)
    s2 = (fx * math.exp(P[3, 0]) / d) ** 2 + 0.3
    col, sig = eff(sc)
    col, sig = col[0], sig[0]
    mu = cam["cx"]
    r = math.ceil(3.0 * math.sqrt(s2 + math.sqrt(0.1)))
    x0 = math.floor((mu - r) / 16)
    outside, inside = 16 * x0 - 1, 16 * x0
    row = int(round(cam["cy"]))
    a_out = min(0.99, sig * math.exp(-0.5 * ((outside - mu) ** 2 + (row - cam["cy"]) ** 2) / s2))
    a_in = min(0.99, sig * math.exp(-0.5 * ((inside - mu) ** 2 + (row - cam["cy"]) ** 2) / s2))
    assert a_out > 1 / 255 and a_in > 1 / 255
    assert img[0, row, outside] == 0.0
    assert img[0, row, inside] == pytest.approx(col[0] * a_in, rel=1e-9)


# ---------------------------------------------------------------- SH basis

def _real_sh_scipy(deg, dirs):
    from scipy.special import sph_harm_y
    x, y, z = dirs.T
    theta = np.arccos(np.clip(z, -1, 1))
    phi = np.arctan2(y, x)
    out = []
    for l in range(deg + 1):
        for m in range(-l, l + 1):
            if m == 0:
                out.append(sph_harm_y(l, 0, theta, phi).real)
            elif m > 0:
                out.append(math.sqrt(2) * (-1) ** m * sph_harm_y(l, m, theta, phi).real)
            else:
                out.append(math.sqrt(2) * (-1) ** m * sph_harm_y(l, -m, theta, phi).imag)
    return np.stack(out, axis=1)


def test_sh_basis_matches_scipy_real_harmonics(oracle):
    rng = np.random.default_rng(0)
    d = rng.normal(size=(200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    np.testing.assert_allclose(oracle.sh_basis(3, d), _real_sh_scipy(3, d), atol=1e-12)


def test_sh_basis_orthonormal_by_quadrature(oracle):
    xg, wg = np.polynomial.legendre.leggauss(12)
    nphi = 24
    phi = 2 * np.pi * np.arange(nphi) / nphi
    ct, ph = np.meshgrid(xg, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    dirs = np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=-1).reshape(-1, 3)
    w = (wg[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).reshape(-1)
    Y = oracle.sh_basis(3, dirs)
    gram = (Y * w[:, None]).T @ Y
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-12)


def _band1_scene(mu, sh0, band1):
    """One small Gaussian at mu with DC sh0 per channel and, in channel c,
    only the band-1 coefficient k = 1 + c set to band1 (k = 1, 2, 3 multiply
    the y, z and x components of the view direction)."""
    sh = np.zeros((1, 4, 3))
    sh[0, 0, :] = sh0
    for c in range(3):
        sh[0, 1 + c, c] = band1
    return I.pack_params(np.asarray([mu], np.float64), np.full((1, 3), math.log(0.05)),
                         np.asarray([[1.0, 0.0, 0.0, 0.0]]), np.asarray([0.5]), sh)


def test_sh_view_direction_degree1_closed_form(oracle):
    """Degree-1 colour in closed form: rgb_c = 0.5 + Y00 sh0_c + sqrt(3/(4 pi))
    sh1_c d_(y, z, x)[c] with d = (mu - eye) / |mu - eye| taken from the eye
    the test placed.  The second eye lies on the other side of the Gaussian,
    which flips every component of d and so every band-1 term: a negated
    direction, or a camera centre taken with the wrong sign, fails here."""
    c1 = math.sqrt(3.0 / (4.0 * math.pi))
    mu = (0.3, -0.2, 0.25)
    sc = _band1_scene(mu, 0.15, 0.6)
    P = sc["params"][:, 0].astype(np.float64)  # the FP32-rounded values the oracle sees
    m = P[0:3]
    cols = []
    for eye in [(2.0, 2.0, 1.5), (-1.5, -2.2, -1.2)]:
        cam = I.pinhole(I.look_at(eye, target=mu), 48, 48)
        pr = oracle.project(sc, cam)
        assert pr["flags"][0] & oracle.G_VISIBLE
        d = m - np.asarray(eye, np.float64)
        d /= np.linalg.norm(d)
        comp = (d[1], d[2], d[0])  # Y_1,-1 ~ y, Y_1,0 ~ z, Y_1,1 ~ x
        expect = np.array([0.5 + Y00 * P[11 + c] + c1 * P[11 + 3 * (1 + c) + c] * comp[c] for c in range(3)])
        # the camera is stored in FP32, so its centre is the eye to ~1e-7
        np.testing.assert_allclose(pr["raw_rgb"][0], expect, rtol=0, atol=2e-6)
        np.testing.assert_allclose(pr["rgb"][0], expect, rtol=0, atol=2e-6)
        cols.append(expect - 0.5 - Y00 * P[11:14])
    # the two eyes see band-1 terms of opposite sign, each well away from zero
    assert np.all(cols[0] * cols[1] < 0) and np.all(np.abs(cols[0]) > 0.05)


@pytest.mark.parametrize("axis,slope", [(0, 1.0), (0, -0.9), (1, 1.1), (0, 0.5)])
def test_guard_band_clamps_the_slope_in_J(oracle, axis, slope):
    """An isotropic Gaussian (Sigma = s^2 I) seen by the axis camera at
    camera-space t = (t_x, t_y, d): Sigma' = s^2 J J^T + 0.3 I with
    J = [[fx/d, 0, -fx u_x/d], [0, fy/d, -fy u_y/d]], u the image-plane slope
    t/d clamped to +-1.3 W/(2 fx) (1.3 H/(2 fy)).  Beyond the guard band the
    conic is that of the clamped slope, its derivative with respect to the
    mean along the clamped axis is zero (only J's slope entries depend on
    it), while mu2D keeps its unclamped derivative fx / d; inside the band
    (slope 0.5) the same derivative is the closed form of the unclamped J."""
    cam = axis_camera(64)
    d, s = 3.0, 0.05
    # camera axes of the axis camera: x = world x, y = -world y, t_z = d - world z
    t_lat = slope * d
    mu = [t_lat, 0.0, 0.0] if axis == 0 else [0.0, -t_lat, 0.0]
    sc = one_scene([mu], [[math.log(s)] * 3], [[1, 0, 0, 0]], [0.0], [(0.5, 0.5, 0.5)])
    P = sc["params"][:, 0].astype(np.float64)
    s2 = math.exp(2.0 * P[3])
    f = cam["fx"] if axis == 0 else cam["fy"]
    size = cam["width"] if axis == 0 else cam["height"]
    lim = 1.3 * size / (2.0 * f)
    t = abs(P[axis]) if axis == 0 else abs(P[1])
    u = t / d
    clamped = u > lim
    assert clamped == (abs(slope) > lim)
    uc = min(u, lim)
    # Sigma' along the lateral axis, and along the other one
    lat = s2 * (f / d) ** 2 * (1.0 + uc * uc) + 0.3
    other = s2 * (cam["fx"] / d) ** 2 + 0.3
    s00, s11 = (lat, other) if axis == 0 else (other, lat)
    pr = oracle.project(sc, cam)
    assert pr["flags"][0] & 32  # 2D quantities computed (in front of znear)
    assert not pr["flags"][0] & oracle.G_MARG_GUARD
    np.testing.assert_allclose(pr["conic"][0], [1.0 / s00, 0.0, 1.0 / s11], rtol=1e-12, atol=1e-15)

    jac, _ = oracle.project_jacobian(sc, cam, 0)
    A_row = 2 if axis == 0 else 4        # the conic entry 1 / Sigma'_lat
    mu_row = 0 if axis == 0 else 1
    wsign = 1.0 if axis == 0 else -1.0   # d t_lat / d world mean
    # d mu2D / d mean: fx / d (camera y = -world y), clamped or not
    assert jac[mu_row, axis] == pytest.approx(wsign * f / d, rel=1e-12)
    dlat_dt = 0.0 if clamped else s2 * (f / d) ** 2 * 2.0 * uc / d * math.copysign(1.0, P[axis])
    expect = -dlat_dt / lat ** 2 * wsign
    if clamped:
        assert jac[A_row, axis] == 0.0
        assert jac[3, axis] == 0.0
    else:
        assert abs(expect) > 1e-3
        assert jac[A_row, axis] == pytest.approx(expect, rel=1e-10)
    # the depth derivative keeps the clamped slope fixed: Sigma'_lat - 0.3 ~ 1 / t_z^2
    dlat_dz = 2.0 * s2 * (f / d) ** 2 * (1.0 + uc * uc) / d
    if not clamped:
        # u = t / t_z also moves with t_z: d(u^2)/d t_z = -2 u^2 / t_z
        dlat_dz += s2 * (f / d) ** 2 * 2.0 * uc * uc / d
    assert jac[A_row, 2] == pytest.approx(-dlat_dz / lat ** 2, rel=1e-10)


# ---------------------------------------------------------------- derivatives

def test_projection_jacobian_matches_finite_differences(oracle):
    sc = I.random_scene(5, 3, 21, extent=0.5)
    cam = I.pinhole(I.look_at((0.4, -2.6, 1.1)), 80, 60)
    p0 = sc["params"].astype(np.float64)
    h = 1e-6
    for g in range(sc["n"]):
        jac, flags = oracle.project_jacobian(sc, cam, g)
        assert flags & oracle.G_VISIBLE
        for pl in range(p0.shape[0]):
            outs = []
            for sgn in (1, -1):
                pp = p0.copy()
                pp[pl, g] += sgn * h
                pr = oracle.project({"params": pp, "n": sc["n"], "deg": 3}, cam)
                outs.append(np.concatenate([pr["mean2d"][g], pr["conic"][g], [pr["opacity"][g]],
                                            pr["rgb"][g]]))
            fd = (outs[0] - outs[1]) / (2 * h)
            np.testing.assert_allclose(jac[:, pl], fd, rtol=1e-5, atol=1e-6 * max(1, np.abs(fd).max()))


@pytest.mark.parametrize("deg,seed", [(0, 1), (3, 2), (3, 3)])
def test_render_gradient_matches_central_differences(oracle, deg, seed):
    sc = I.random_scene(8, deg, seed, extent=0.4, log_scale=(-2.6, -1.6))
    cam = I.pinhole(I.look_at((0.3, -2.5, 0.8)), 32, 32, bg=(0.1, 0.2, 0.3))
    rng = np.random.default_rng(seed)
    dimg = rng.normal(size=(3, 32, 32))
    grad = oracle.render_grad(sc, [cam], [dimg])
    p0 = sc["params"].astype(np.float64)

    def L(p):
        img, _, _, _ = oracle.render({"params": p, "n": sc["n"], "deg": deg}, cam)
        return float(np.sum(img * dimg))

    h = 1e-6
    fd = np.zeros_like(p0)
    for pl in range(p0.shape[0]):
        for g in range(sc["n"]):
            pp, pm = p0.copy(), p0.copy()
            pp[pl, g] += h
            pm[pl, g] -= h
            fd[pl, g] = (L(pp) - L(pm)) / (2 * h)
    scale = np.abs(grad).max()
    assert scale > 0
    assert np.abs(fd - grad).max() <= 1e-6 * scale


def test_two_view_gradient_is_sum_of_views(oracle):
    sc = I.random_scene(10, 1, 4, extent=0.4)
    cams = [I.pinhole(I.look_at(e), 32, 24) for e in [(0.3, -2.5, 0.8), (2.0, 1.0, -1.0)]]
    rng = np.random.default_rng(1)
    dimgs = [rng.normal(size=(3, 24, 32)) for _ in cams]
    both = oracle.render_grad(sc, cams, dimgs)
    sep = sum(oracle.render_grad(sc, [c], [d]) for c, d in zip(cams, dimgs))
    np.testing.assert_allclose(both, sep, rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------- invariants

def test_rotating_scene_and_camera_together_leaves_image(oracle):
    from scipy.spatial.transform import Rotation
    sc = I.random_scene(40, 0, 9, extent=0.6)
    cam = I.pinhole(I.look_at((0.3, -2.7, 0.9)), 64, 48)
    Rq = Rotation.from_euler("xyz", [0.4, -0.9, 1.3])
    Q = Rq.as_matrix()
    u = I.unpack_params(sc)
    q_xyzw = np.concatenate([u["quats"][:, 1:], u["quats"][:, :1]], axis=1)
    qn = (Rq * Rotation.from_quat(q_xyzw)).as_quat()
    quats = np.concatenate([qn[:, 3:], qn[:, :3]], axis=1)
    p2 = sc["params"].astype(np.float64)          # rotated copy kept in FP64
    n = sc["n"]
    p2[0:3, :n] = (u["means"].astype(np.float64) @ Q.T).T
    p2[6:10, :n] = quats.T
    sc2 = {"params": p2, "n": n, "deg": 0}
    sc1 = dict(sc)
    sc1["params"] = sc["params"].astype(np.float64)
    cam2 = dict(cam)
    M = np.eye(4)
    M[:3, :3] = Q.T
    cam2["viewmat"] = cam["viewmat"] @ M
    img1, _, m1, _ = oracle.render(sc1, cam)
    img2, _, m2, _ = oracle.render(sc2, cam2)
    ok = ~(m1 | m2)
    assert ok.mean() > 0.99
    np.testing.assert_allclose(img1[:, ok], img2[:, ok], atol=1e-9)


def test_quaternion_sign_and_scale_do_not_matter(oracle):
    sc = I.random_scene(30, 2, 13, extent=0.6)
    cam = I.pinhole(I.look_at((0.3, -2.7, 0.9)), 48, 48)
    sc2 = {"params": sc["params"].copy(), "n": sc["n"], "deg": 2}
    sc2["params"][6:10] *= -2.0          # exact in FP32
    a, _, _, _ = oracle.render(sc, cam)
    b, _, _, _ = oracle.render(sc2, cam)
    np.testing.assert_allclose(a, b, atol=1e-10)


def test_invariants_on_sphere_scene(oracle):
    sc = I.sphere_scene()
    cam = I.sphere_camera()
    img, tf, mg, _ = oracle.render(sc, cam)
    assert np.all(tf >= 1e-4) and np.all(tf <= 1.0)
    assert np.all(img >= 0.0)
    assert mg.mean() < 0.01
    pr = oracle.project(sc, cam)
    # rect equals the brute-force set of tiles satisfying the two edge inequalities
    gw = gh = 16
    tx = np.arange(gw)
    for g in range(0, sc["n"], 97):
        if not pr["flags"][g] & oracle.G_VISIBLE:
            continue
        mx, my = pr["mean2d"][g]
        r = pr["radius"][g]
        inx = (16 * tx + 16 > mx - r) & (16 * tx + 1 <= mx + r)
        iny = (16 * tx + 16 > my - r) & (16 * tx + 1 <= my + r)
        x0, x1, y0, y1 = pr["rect"][g]
        assert list(np.nonzero(inx)[0]) == list(range(x0, x1))
        assert list(np.nonzero(iny)[0]) == list(range(y0, y1))
        assert pr["tiles"][g] == inx.sum() * iny.sum()
    # transparent scene -> background
    sc0 = {"params": sc["params"].copy(), "n": sc["n"], "deg": 0}
    sc0["params"][10] = -60.0
    cam_bg = dict(cam)
    cam_bg["bg"] = (0.25, 0.5, 0.75)
    img0, tf0, _, _ = oracle.render(sc0, cam_bg)
    for c in range(3):
        assert np.all(img0[c] == 0.25 * (c + 1))
    assert np.all(tf0 == 1.0)


def test_depth_is_the_specified_fp32_evaluation(oracle):
    sc = I.random_scene(200, 0, 17, extent=0.8)
    cam = I.pinhole(I.look_at((1.3, -2.2, 0.7)), 64, 64)
    pr = oracle.project(sc, cam)
    V = cam["viewmat"].astype(np.float32)
    m = sc["params"][0:3, :sc["n"]].astype(np.float32)
    ab = V[2, 0] * m[0] + V[2, 1] * m[1]
    d = (ab + V[2, 2] * m[2]) + V[2, 3]
    np.testing.assert_array_equal(pr["depth"].astype(np.float32), d.astype(np.float32))


# ---------------------------------------------------------------- loss, Adam

def test_l1_closed_form(oracle):
    x = np.array([1.0, 2.0, 3.0, 4.0])
    y = np.array([1.5, 2.0, 1.0, 5.0])
    loss, g = oracle.l1(x, y)
    assert loss == pytest.approx((0.5 + 0 + 2 + 1) / 4)
    np.testing.assert_array_equal(g, [-0.25, 0.0, 0.25, -0.25])


def test_adam_first_step_closed_form(oracle):
    rng = np.random.default_rng(0)
    P, n = 4, 8
    p = rng.normal(size=(P, n))
    g = rng.normal(size=(P, n))
    lr = np.array([1e-3, 2e-3, 5e-2, 1e-4])
    p1 = p.copy()
    oracle.adam(p1, g, np.zeros((P, n)), np.zeros((P, n)), lr, 1)
    np.testing.assert_allclose(p1, p - lr[:, None] * g / (np.abs(g) + 1e-15), rtol=1e-12)


def test_adam_matches_torch_over_steps(oracle):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    P, n = 3, 10
    p0 = rng.normal(size=(P, n))
    lr = [1e-2, 3e-3, 5e-2]
    tp = [torch.tensor(p0[i], dtype=torch.float64, requires_grad=True) for i in range(P)]
    opt = torch.optim.Adam([{"params": [tp[i]], "lr": lr[i]} for i in range(P)],
                           betas=(0.9, 0.999), eps=1e-15)
    p, m, v = p0.copy(), np.zeros((P, n)), np.zeros((P, n))
    for step in range(1, 6):
        g = rng.normal(size=(P, n))
        for i in range(P):
            tp[i].grad = torch.tensor(g[i], dtype=torch.float64)
        opt.step()
        oracle.adam(p, g, m, v, np.array(lr), step)
    np.testing.assert_allclose(p, np.stack([t.detach().numpy() for t in tp]), rtol=1e-12, atol=1e-15)


def test_visible_only_adam_matches_torch_sparse_adam(oracle):
    """Visible-only Adam: invisible Gaussians keep parameters and moments
    exactly; visible ones equal torch.optim.SparseAdam's lazy update (moments
    touched only where the gradient is present, bias correction by the
    global step) and the dense step of the same state."""
    rng = np.random.default_rng(11)
    P, n = 14, 37
    lr = rng.uniform(1e-4, 1e-2, size=P)
    p = rng.normal(size=(P, n))
    m = np.zeros((P, n))
    v = np.zeros((P, n))
    tp = [torch.tensor(p[k].copy(), requires_grad=True) for k in range(P)]
    opts = [torch.optim.SparseAdam([tp[k]], lr=float(lr[k]), betas=(0.9, 0.999), eps=1e-15) for k in range(P)]
    for step in range(1, 5):
        vis = (rng.uniform(size=n) < 0.6).astype(np.uint8)
        g = rng.normal(size=(P, n)) * vis
        before = (p.copy(), m.copy(), v.copy())
        dense = (p.copy(), g.copy(), m.copy(), v.copy())
        oracle.adam(dense[0], dense[1], dense[2], dense[3], lr, step)
        oracle.adam_visible(p, g, m, v, lr, step, vis)
        hid = vis == 0
        assert np.array_equal(p[:, hid], before[0][:, hid])
        assert np.array_equal(m[:, hid], before[1][:, hid]) and np.array_equal(v[:, hid], before[2][:, hid])
        np.testing.assert_allclose(p[:, ~hid], dense[0][:, ~hid], rtol=1e-14, atol=1e-15)
        idx = np.nonzero(vis)[0]
        for k in range(P):
            tp[k].grad = torch.sparse_coo_tensor(torch.tensor(idx)[None], torch.tensor(g[k, idx]), (n,))
            opts[k].step()
    for k in range(P):
        np.testing.assert_allclose(p[k], tp[k].detach().numpy(), rtol=1e-9, atol=1e-12)
