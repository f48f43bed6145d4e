"""Seeded synthetic workloads: Gaussian sets, orbit cameras and perturbations.

This module only builds inputs. It holds none of the rasterizer's arithmetic
(projection, compositing, gradients, Adam); both the CUDA path and the CPU
oracle consume what it returns.

The paper initialises its Gaussians from isosurface point clouds extracted
from volume data, with no image-based reconstruction, and trains them against
views on a structured camera orbit (Section III, "Method Overview"); its
workloads are about 4M points (Kingsnake) and about 18.18M points (Miranda) at
512^2..2048^2 with 448 views (Section IV). The datasets are not available, so
the generators below produce isosurfaces of seeded analytic fields with the
same point counts.

Parameter layout (one float32 array of shape [P, stride], "SoA planes"):
    planes 0-2   mean x, y, z
    planes 3-5   log-scale s0, s1, s2
    planes 6-9   rotation quaternion w, x, y, z (not necessarily unit)
    plane  10    opacity logit
    planes 11..  SH coefficients, coefficient-major: plane 11 + 3*k + c holds
                 coefficient k (k = l*l + l + m) of colour channel c
P = 11 + 3*(deg+1)^2; stride >= n is a multiple of 4 (padding is zero).

Camera (dict): 'viewmat' 4x4 float64 world->camera (rows: right, down,
forward; camera looks down +z), 'fx', 'fy', 'cx', 'cy', 'width', 'height',
'znear', 'bg' (3 floats).
"""
from __future__ import annotations

import math

import numpy as np

N_BASE_PLANES = 11


def n_sh_coeffs(deg: int) -> int:
    return (deg + 1) * (deg + 1)


def n_planes(deg: int) -> int:
    return N_BASE_PLANES + 3 * n_sh_coeffs(deg)


def padded_stride(n: int) -> int:
    return max(4, (n + 3) // 4 * 4)


def pack_params(means, log_scales, quats, opacity_logits, sh, stride=None):
    """Pack per-Gaussian arrays into the [P, stride] float32 plane layout.

    means [n,3], log_scales [n,3], quats [n,4] (w,x,y,z), opacity_logits [n],
    sh [n, K, 3].
    """
    n = means.shape[0]
    k = sh.shape[1]
    deg = int(round(math.sqrt(k))) - 1
    assert n_sh_coeffs(deg) == k
    stride = padded_stride(n) if stride is None else stride
    out = np.zeros((n_planes(deg), stride), dtype=np.float32)
    out[0:3, :n] = means.T
    out[3:6, :n] = log_scales.T
    out[6:10, :n] = quats.T
    out[10, :n] = opacity_logits
    out[11:, :n] = sh.reshape(n, 3 * k).T
    return {"params": out, "n": n, "deg": deg}


def unpack_params(scene):
    p, n, deg = scene["params"], scene["n"], scene["deg"]
    k = n_sh_coeffs(deg)
    return dict(means=p[0:3, :n].T.copy(), log_scales=p[3:6, :n].T.copy(),
                quats=p[6:10, :n].T.copy(), opacity_logits=p[10, :n].copy(),
                sh=p[11:, :n].T.reshape(n, k, 3).copy())


# ---------------------------------------------------------------- cameras

def look_at(eye, target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0)):
    """World->camera 4x4 matrix; camera x = right, y = down, z = forward."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    up = np.asarray(up, np.float64)
    right = np.cross(f, up)
    if np.linalg.norm(right) < 1e-9:          # looking along `up`
        right = np.cross(f, np.array([0.0, 1.0, 0.0]))
        if np.linalg.norm(right) < 1e-9:
            right = np.cross(f, np.array([1.0, 0.0, 0.0]))
    right /= np.linalg.norm(right)
    down = np.cross(f, right)
    rot = np.stack([right, down, f])
    m = np.eye(4)
    m[:3, :3] = rot
    m[:3, 3] = -rot @ eye
    return m


def _f32(x):
    return float(np.float32(x))


def pinhole(viewmat, width, height, fov_x_deg=60.0, znear=0.2, bg=(0.0, 0.0, 0.0)):
    """Camera record.  Every real number is rounded to FP32 here, so that an
    FP32 consumer and an FP64 consumer see the same camera."""
    fx = _f32(width / (2.0 * math.tan(math.radians(fov_x_deg) / 2.0)))
    vm = np.asarray(viewmat, np.float64).astype(np.float32).astype(np.float64)
    return {"viewmat": vm, "fx": fx, "fy": fx,
            "cx": _f32((width - 1) / 2.0), "cy": _f32((height - 1) / 2.0),
            "width": int(width), "height": int(height), "znear": _f32(znear),
            "bg": tuple(_f32(b) for b in bg)}


def orbit_cameras(n_az, n_el, radius, width, height, fov_x_deg=60.0,
                  el_range_deg=(-75.0, 75.0), bg=(0.0, 0.0, 0.0)):
    """Structured orbit: n_az azimuths x n_el evenly spaced elevations."""
    cams = []
    lo, hi = el_range_deg
    for j in range(n_el):
        el = math.radians(lo + (hi - lo) * (j + 0.5) / n_el)
        for i in range(n_az):
            az = 2.0 * math.pi * i / n_az
            eye = radius * np.array([math.cos(el) * math.cos(az),
                                     math.cos(el) * math.sin(az), math.sin(el)])
            cams.append(pinhole(look_at(eye), width, height, fov_x_deg, bg=bg))
    return cams


def random_orbit_camera(rng, radius, width, height, fov_x_deg=60.0):
    """Camera at a uniformly random point of the sphere, looking at the origin."""
    v = rng.normal(size=3)
    v /= np.linalg.norm(v)
    return pinhole(look_at(radius * v), width, height, fov_x_deg)


# ---------------------------------------------------------------- perturbation

def perturb(scene, seed, frac=0.05):
    """Seeded +-frac perturbation: p' = p(1+frac*u) for p != 0, p + frac*u for p == 0."""
    rng = np.random.default_rng(seed)
    p = scene["params"]
    n = scene["n"]
    u = rng.uniform(-1.0, 1.0, size=(p.shape[0], n)).astype(np.float64)
    x = p[:, :n].astype(np.float64)
    y = np.where(x != 0.0, x * (1.0 + frac * u), x + frac * u)
    out = p.copy()
    out[:, :n] = y.astype(np.float32)
    return {"params": out, "n": n, "deg": scene["deg"]}


# ---------------------------------------------------------------- helpers

_LIGHT = np.array([1.0, 1.0, 1.0]) / math.sqrt(3.0)
# The DC coefficient that reproduces a grey level c under the SH colour rule
# rgb = Y00 * sh0 + 0.5 with Y00 = 1 / (2 sqrt(pi)); this is how the seeded
# scenes choose their base colour.
_DC_FROM_GREY = 2.0 * math.sqrt(math.pi)


def _lambert_dc(normals):
    c = 0.1 + 0.9 * np.maximum(0.0, normals @ _LIGHT)
    return (c - 0.5) * _DC_FROM_GREY


def _quat_z_to(normals):
    """Quaternions (w,x,y,z) rotating +z onto each unit normal."""
    w = 1.0 + normals[:, 2]
    q = np.stack([w, -normals[:, 1], normals[:, 0], np.zeros_like(w)], axis=1)
    bad = w < 1e-6
    q[bad] = np.array([0.0, 1.0, 0.0, 0.0])
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def knn_log_scale(points, k=3):
    """log sqrt(mean squared distance to the k nearest neighbours)."""
    from scipy.spatial import cKDTree
    tree = cKDTree(points)
    d, _ = tree.query(points, k=k + 1, workers=-1)
    msq = np.mean(d[:, 1:] ** 2, axis=1)
    msq = np.maximum(msq, 1e-14)
    return 0.5 * np.log(msq)


def _surface_scene(points, normals, deg, seed, flatten=0.3, opacity_logit=2.0,
                   sh_rest_std=0.02):
    """Reference Gaussian set for an isosurface point cloud: one Gaussian per
    point, flattened along the surface normal, Lambertian DC colour."""
    rng = np.random.default_rng(seed + 1000)
    n = points.shape[0]
    ls = knn_log_scale(points)
    log_scales = np.stack([ls, ls, ls + math.log(flatten)], axis=1)
    quats = _quat_z_to(normals)
    k = n_sh_coeffs(deg)
    sh = np.zeros((n, k, 3))
    sh[:, 0, :] = _lambert_dc(normals)[:, None]
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, sh_rest_std, size=(n, k - 1, 3))
    return pack_params(points, log_scales, quats, np.full(n, opacity_logit), sh)


# ---------------------------------------------------------------- config 1

def sphere_scene(n=10_000, seed=1):
    """n means uniform on the unit sphere, isotropic log-scale -4, identity
    rotation, opacity logit 0, SH degree 0 grey from Lambertian shading."""
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    sh = _lambert_dc(v)[:, None, None] * np.ones((1, 1, 3))
    quats = np.tile(np.array([1.0, 0.0, 0.0, 0.0]), (n, 1))
    return pack_params(v, np.full((n, 3), -4.0), quats, np.zeros(n), sh)


def sphere_camera(width=256, height=256, distance=3.0):
    return pinhole(look_at((0.0, 0.0, distance), up=(0.0, 1.0, 0.0)), width, height)


# ---------------------------------------------------------------- field sampler
#
# The analytic fields are evaluated with torch in float64 on `device` ("cuda"
# when available for the large scenes, "cpu" otherwise); random draws come
# from numpy's seeded generator, so a scene depends only on its seed (up to
# the last bits of the Newton iterations on different devices).

def _device(device):
    import torch
    if device is None:
        device = "cuda" if torch.cuda.is_available() else "cpu"
    return torch.device(device)


def _chunked(fn, x, chunk):
    import torch
    outs = [fn(x[i:i + chunk]) for i in range(0, x.shape[0], chunk)]
    if isinstance(outs[0], tuple):
        return tuple(torch.cat([o[j] for o in outs]) for j in range(len(outs[0])))
    return torch.cat(outs)


def _newton_surface(fg, x, iso, steps):
    for _ in range(steps):
        f, g = fg(x)
        x = x - ((f - iso) / (g * g).sum(dim=1).clamp_min(1e-30))[:, None] * g
    return x


def _sample_isosurface(fg, lo, hi, iso, n, seed, res=96, jitter=0.0, device=None):
    """Exactly n points on {field = iso} inside the box [lo, hi]^3.

    fg(x) -> (field, gradient) on a torch float64 [m, 3] tensor.  Lattice
    cells whose corners straddle the level are found on a res^3 grid; cells
    are drawn uniformly (seeded) and a uniform point inside each is
    Newton-projected onto the level set, so the density is close to uniform
    per unit area.  Points that do not converge or leave their cell's
    neighbourhood are redrawn.  The points are returned in the order a
    contour filter emits them: by the grid cell that holds them, x fastest,
    then y, then z (the draws themselves do not depend on this order).
    """
    import torch
    dev = _device(device)
    rng = np.random.default_rng(seed)
    h = (hi - lo) / res
    ax = torch.tensor(lo + h * np.arange(res + 1), dtype=torch.float64, device=dev)
    gx, gy = torch.meshgrid(ax, ax, indexing="ij")
    cells = []
    prev = None
    for iz in range(res + 1):
        pts = torch.stack([gx.reshape(-1), gy.reshape(-1), torch.full_like(gx.reshape(-1), float(ax[iz]))], 1)
        sgn = (fg(pts)[0] >= iso).reshape(res + 1, res + 1)
        if prev is not None:
            c = torch.stack([prev[:-1, :-1], prev[1:, :-1], prev[:-1, 1:], prev[1:, 1:],
                             sgn[:-1, :-1], sgn[1:, :-1], sgn[:-1, 1:], sgn[1:, 1:]])
            straddle = c.any(0) & ~c.all(0)
            ix, iy = torch.nonzero(straddle, as_tuple=True)
            cells.append(np.stack([ix.cpu().numpy(), iy.cpu().numpy(), np.full(ix.numel(), iz - 1)], 1))
        prev = sgn
    cells = np.concatenate(cells, axis=0)
    if cells.shape[0] == 0:
        raise ValueError("isosurface does not cross the domain")
    out, have = [], 0
    while have < n:
        m = int((n - have) * 1.3) + 64
        pick = cells[rng.integers(0, cells.shape[0], size=m)]
        x0 = lo + h * (pick + rng.uniform(0.0, 1.0, size=(m, 3)))
        jit = rng.normal(0.0, jitter, size=(m, 3)) if jitter > 0.0 else None
        x0t = torch.from_numpy(x0).to(dev)
        x = _newton_surface(fg, x0t, iso, 6)
        if jit is not None:
            x = _newton_surface(fg, x + torch.from_numpy(jit).to(dev), iso, 4)
        f, _ = fg(x)
        ok = ((f - iso).abs() < 1e-7) & torch.isfinite(x).all(1)
        ok &= (x - x0t).norm(dim=1) < 2.0 * h * math.sqrt(3.0)
        ok &= ((x >= lo) & (x <= hi)).all(1)
        x = x[ok].cpu().numpy()
        out.append(x)
        have += x.shape[0]
    pts = np.concatenate(out, axis=0)[:n]
    cell = np.clip(np.floor((pts - lo) / h).astype(np.int64), 0, res - 1)
    order = np.argsort((cell[:, 2] * res + cell[:, 1]) * res + cell[:, 0], kind="stable")
    return pts[order]


# ---------------------------------------------------------------- config 2

def _gyroid_fg(x):
    import torch
    sx, cx = torch.sin(x[:, 0]), torch.cos(x[:, 0])
    sy, cy = torch.sin(x[:, 1]), torch.cos(x[:, 1])
    sz, cz = torch.sin(x[:, 2]), torch.cos(x[:, 2])
    f = sx * cy + sy * cz + sz * cx
    g = torch.stack([cx * cy - sz * sx, -sx * sy + cy * cz, -sy * sz + cz * cx], 1)
    return f, g


def gyroid_scene(n=500_000, seed=3, deg=3, res=96, device=None):
    """Gaussians on the gyroid sin x cos y + sin y cos z + sin z cos x = 0
    over [-2pi, 2pi]^3 (Newton-projected samples with N(0, 0.01) jitter)."""
    import torch
    lo, hi = -2.0 * math.pi, 2.0 * math.pi
    pts = _sample_isosurface(_gyroid_fg, lo, hi, 0.0, n, seed, res=res, jitter=0.01, device=device)
    _, g = _gyroid_fg(torch.from_numpy(pts))
    g = g.numpy()
    nrm = g / np.linalg.norm(g, axis=1, keepdims=True)
    return _surface_scene(pts, nrm, deg, seed)


# ---------------------------------------------------------------- config 3

class BlobField:
    """f(x) = sum_k a_k exp(-1/2 (x-c_k)^T S_k^-1 (x-c_k)) with seeded random
    amplitudes U(0.6,1), centres U(-0.8,0.8)^3, rotations and axis std-devs
    U(0.02,0.15); the [-1,1]^3 box stands for the 512^3 volume.  Terms
    beyond 4.5 standard deviations along every axis are left out (part of the
    field's definition)."""

    def __init__(self, seed=4, n_blobs=200):
        rng = np.random.default_rng(seed)
        self.a = rng.uniform(0.6, 1.0, size=n_blobs)
        self.c = rng.uniform(-0.8, 0.8, size=(n_blobs, 3))
        q = rng.normal(size=(n_blobs, 4))
        q /= np.linalg.norm(q, axis=1, keepdims=True)
        w, x, y, z = q.T
        rot = np.stack([
            np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
            np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
            np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
        ], axis=1)
        sd = rng.uniform(0.02, 0.15, size=(n_blobs, 3))
        self.prec = np.einsum("kij,kj,klj->kil", rot, 1.0 / sd ** 2, rot)
        self.reach = 4.5 * sd.max(axis=1)
        self._t = {}

    def _tensors(self, dev):
        import torch
        if dev not in self._t:
            self._t[dev] = tuple(torch.from_numpy(np.ascontiguousarray(v)).to(dev)
                                 for v in (self.a, self.c, self.prec, self.reach))
        return self._t[dev]

    def fg(self, x):
        """(field, gradient) at points x (torch float64 [m, 3])."""
        import torch
        a, c, prec, reach = self._tensors(x.device)

        def one(xc):
            d = xc[:, None, :] - c[None]                       # [m, K, 3]
            near = (d.abs() < reach[None, :, None]).all(-1)     # [m, K]
            pd = torch.einsum("mkj,kij->mki", d, prec)
            e = a[None] * torch.exp(-0.5 * (d * pd).sum(-1)) * near
            return e.sum(1), -(e[..., None] * pd).sum(1)
        return _chunked(one, x, 1 << 16)


def blobs_scene(n=4_000_000, seed=4, deg=3, res=128, iso=0.5, device=None):
    """Gaussians on the 0.5 level of a 200-blob field (Kingsnake-scale stand-in)."""
    import torch
    fld = BlobField(seed)
    pts = _sample_isosurface(fld.fg, -1.0, 1.0, iso, n, seed, res=res, device=device)
    _, g = _chunked(fld.fg, torch.from_numpy(pts).to(_device(device)), 1 << 16)
    g = g.cpu().numpy()
    nrm = -g / np.linalg.norm(g, axis=1, keepdims=True)
    return _surface_scene(pts, nrm, deg, seed)


# ---------------------------------------------------------------- config 4

class NoiseField:
    """Fractal value noise: f(x) = sum_{o<6} 0.5^o n(4 * 2^o * (x + 1) / 2),
    n = trilinear interpolation (smoothstep weights) of seeded lattice values
    in [-1, 1]; the [-1,1]^3 box stands for the 1024^3 volume."""

    def __init__(self, seed=5, octaves=6, base=4.0, lacunarity=2.0, gain=0.5):
        self.seed, self.octaves, self.base, self.lac, self.gain = seed, octaves, base, lacunarity, gain

    def _lattice(self, ix, iy, iz, o):
        import torch
        h = (ix * 73856093) ^ (iy * 19349663) ^ (iz * 83492791) ^ ((self.seed * 2654435761 + o * 97) & 0x7FFFFFFF)
        h = (h ^ (h >> 13)) * 1274126177
        h = h ^ (h >> 16)
        return (h & 0xFFFFFF).to(torch.float64) / float(0x7FFFFF) - 1.0

    def fg(self, x):
        import torch
        f = torch.zeros(x.shape[0], dtype=torch.float64, device=x.device)
        g = torch.zeros_like(x)
        for o in range(self.octaves):
            freq = self.base * self.lac ** o
            amp = self.gain ** o
            u = (x + 1.0) * 0.5 * freq
            i0 = torch.floor(u)
            t = u - i0
            w = t * t * (3.0 - 2.0 * t)
            dw = 6.0 * t * (1.0 - t) * 0.5 * freq
            ii = i0.to(torch.int64)
            val = torch.zeros_like(f)
            dval = torch.zeros_like(g)
            for cx in (0, 1):
                for cy in (0, 1):
                    for cz in (0, 1):
                        lv = self._lattice(ii[:, 0] + cx, ii[:, 1] + cy, ii[:, 2] + cz, o)
                        wx = w[:, 0] if cx else 1.0 - w[:, 0]
                        wy = w[:, 1] if cy else 1.0 - w[:, 1]
                        wz = w[:, 2] if cz else 1.0 - w[:, 2]
                        sx = 1.0 if cx else -1.0
                        sy = 1.0 if cy else -1.0
                        sz = 1.0 if cz else -1.0
                        val = val + lv * wx * wy * wz
                        dval[:, 0] += lv * sx * dw[:, 0] * wy * wz
                        dval[:, 1] += lv * sy * dw[:, 1] * wx * wz
                        dval[:, 2] += lv * sz * dw[:, 2] * wx * wy
            f = f + amp * val
            g = g + amp * dval
        return f, g


def noise_scene(n=18_000_000, seed=5, deg=3, res=256, device=None):
    """Gaussians on the zero level of 6-octave fractal value noise (Miranda-scale stand-in)."""
    import torch
    fld = NoiseField(seed)
    fg = lambda x: _chunked(fld.fg, x, 1 << 20)
    pts = _sample_isosurface(fg, -1.0, 1.0, 0.0, n, seed, res=res, device=device)
    _, g = fg(torch.from_numpy(pts).to(_device(device)))
    g = g.cpu().numpy()
    nrm = g / np.linalg.norm(g, axis=1, keepdims=True)
    return _surface_scene(pts, nrm, deg, seed)


# ---------------------------------------------------------------- generic small scenes

def random_scene(n, deg, seed, extent=1.0, log_scale=(-3.5, -2.0), opacity=(-2.0, 3.0)):
    """Gaussians with random means in a cube, random anisotropic scales,
    random rotations, opacities and SH colours (for tests)."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-extent, extent, size=(n, 3))
    ls = rng.uniform(log_scale[0], log_scale[1], size=(n, 3))
    q = rng.normal(size=(n, 4))
    o = rng.uniform(opacity[0], opacity[1], size=n)
    k = n_sh_coeffs(deg)
    sh = rng.normal(0.0, 0.3, size=(n, k, 3))
    sh[:, 0, :] = rng.uniform(-1.0, 1.5, size=(n, 3))
    return pack_params(means, ls, q, o, sh)
