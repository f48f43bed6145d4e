"""Point-cloud initialisation on the GPU against the oracle (GPU only):
isosurface edge crossings of a sampled volume (count, order, points,
normals) and the initial Gaussians (means, k-nearest-neighbour scales,
rotations, opacity, colour) of random and isosurface point sets."""
import math

import numpy as np
import pytest
import torch

from oracle import init as OI
from paper_2509_05216_gb300 import gs, inputs

pytestmark = pytest.mark.gpu


def sampled_field(n, seed):
    """A smooth random field (a few Gaussian bumps) on an n^3 grid in [-1, 1]^3."""
    rng = np.random.default_rng(seed)
    ax = np.linspace(-1.0, 1.0, n)
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    f = np.zeros_like(x)
    for _ in range(6):
        c = rng.uniform(-0.6, 0.6, 3)
        s = rng.uniform(0.2, 0.5)
        f += np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) / (2 * s * s))
    return f.astype(np.float32), ax[1] - ax[0]


def test_crossings_match_oracle():
    vol, h = sampled_field(29, 1)
    ctx = gs.Context(0)
    iso = 0.5
    pts, nrm = ctx.gs_iso_crossings(torch.from_numpy(vol).cuda(), iso, (-1.0, -1.0, -1.0), (h, h, h))
    rp, rn = OI.iso_crossings(vol, iso, (-1.0, -1.0, -1.0), (h, h, h))
    assert pts.shape[0] == rp.shape[0] > 500
    np.testing.assert_allclose(pts.cpu().numpy(), rp, rtol=0, atol=2e-6)
    cos = np.sum(nrm.cpu().numpy().astype(np.float64) * rn, axis=1)
    assert cos.min() > 1 - 1e-5
    # a level no sample reaches: no crossings
    p0, _ = ctx.gs_iso_crossings(torch.from_numpy(vol).cuda(), 99.0, (-1.0, -1.0, -1.0), (h, h, h))
    assert p0.shape[0] == 0
    ctx.close()


def test_crossings_capacity_is_reported():
    vol, h = sampled_field(17, 2)
    ctx = gs.Context(0)
    v = torch.from_numpy(vol).cuda()
    import ctypes
    o = (ctypes.c_float * 3)(-1.0, -1.0, -1.0)
    hh = (ctypes.c_float * 3)(h, h, h)
    cnt = ctypes.c_int64()
    buf = torch.empty((4, 3), device="cuda")
    st = ctx.L.gs_iso_crossings(ctx.h, ctypes.c_void_p(v.data_ptr()), 17, 17, 17, 0.5, o, hh,
                                ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(buf.data_ptr()), 4, ctypes.byref(cnt))
    assert st == gs.GS_ECAPACITY and cnt.value > 4
    ctx.close()


def marginal_ties(points, k=3):
    """Points whose k-th and (k+1)-th neighbour distances nearly tie (FP32
    may then pick either)."""
    from scipy.spatial import cKDTree
    p = np.asarray(points, np.float64)
    d, _ = cKDTree(p).query(p, k=k + 2)
    return np.abs(d[:, k + 1] - d[:, k]) <= 1e-5 * np.maximum(d[:, k], 1e-12)


@pytest.mark.parametrize("kind", ["random", "surface"])
def test_init_gaussians_match_oracle(kind):
    rng = np.random.default_rng(3)
    if kind == "random":
        n = 5003
        pts = rng.uniform(-1, 1, size=(n, 3)).astype(np.float32)
        nrm = rng.normal(size=(n, 3))
        nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
        nrm[0] = [0.0, 0.0, -1.0]
        nrm = nrm.astype(np.float32)
        sel = None
        m = n
    else:  # crossings of a sampled field, a seeded subset
        vol, h = sampled_field(65, 4)
        ctx0 = gs.Context(0)
        tp, tn = ctx0.gs_iso_crossings(torch.from_numpy(vol).cuda(), 0.5, (-1.0, -1.0, -1.0), (h, h, h))
        ctx0.close()
        pts, nrm = tp.cpu().numpy(), tn.cpu().numpy()
        m = pts.shape[0]
        n = m // 2
        sel = np.sort(rng.choice(m, size=n, replace=False)).astype(np.int64)
    deg = 3
    P = 11 + 3 * (deg + 1) ** 2
    out = torch.zeros((P, inputs.padded_stride(n)), device="cuda")
    ctx = gs.Context(0)
    ctx.gs_init_gaussians(torch.from_numpy(pts).cuda(), torch.from_numpy(nrm).cuda(), out, n, deg,
                          None if sel is None else torch.from_numpy(sel).cuda(), flatten=0.3, opacity_logit=2.0)
    ctx.gs_sync()
    got = out.cpu().numpy()[:, :n].astype(np.float64)
    sp = pts if sel is None else pts[sel]
    sn = nrm if sel is None else nrm[sel]
    ref = OI.init_gaussians(sp, sn, 0.3, 2.0, deg)
    np.testing.assert_array_equal(got[0:3], sp.T.astype(np.float64))
    ok = ~marginal_ties(sp)
    assert ok.mean() > 0.99
    np.testing.assert_allclose(got[3:6][:, ok], ref[3:6][:, ok], rtol=0, atol=2e-5)
    np.testing.assert_allclose(got[6:11], ref[6:11], rtol=0, atol=2e-6)
    np.testing.assert_allclose(got[11:], ref[11:], rtol=0, atol=2e-6)
    ctx.close()


def test_init_rejects_bad_arguments():
    ctx = gs.Context(0)
    pts = torch.zeros((3, 3), device="cuda")
    out = torch.zeros((59, 4), device="cuda")
    with pytest.raises(gs.GsError) as e:
        ctx.gs_init_gaussians(pts, pts, out, 3, 3)
    assert e.value.status == gs.GS_EINVAL
    pts = torch.zeros((8, 3), device="cuda")  # all at one point: no box
    out = torch.zeros((59, 8), device="cuda")
    with pytest.raises(gs.GsError) as e:
        ctx.gs_init_gaussians(pts, pts, out, 8, 3)
    assert e.value.status == gs.GS_EINVAL
    ctx.close()
