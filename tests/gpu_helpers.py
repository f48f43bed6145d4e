"""Helpers shared by the GPU parity tests: run the CUDA path through the C
ABI and recompute integer binning on the CPU from the GPU's own FP32 values."""
import numpy as np
import torch

from paper_2509_05216_gb300 import gs


def run_forward(ctx, scene, cams):
    p = torch.from_numpy(scene["params"]).cuda()
    ctx.gs_project(p, scene["n"], scene["deg"], cams)
    ctx.gs_bin_sort()
    _, total = gs.image_offsets(cams)
    img = torch.full((total,), float("nan"), device="cuda")
    ctx.gs_raster_fwd(img)
    ctx.gs_sync()
    return p, img


def to_dev_images(arrs):
    return torch.cat([torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).reshape(-1)
                      for a in arrs]).cuda()


def cpu_rect(mx, my, r, W, H):
    """Tile rect from FP32 mean and integer radius, in FP32 arithmetic."""
    f = np.float32
    gw, gh = (W + 15) // 16, (H + 15) // 16
    r32 = r.astype(np.float32)
    r15 = (r + 15).astype(np.float32)
    x0 = np.clip(np.floor((mx.astype(f) - r32) * f(0.0625)), 0, gw).astype(np.int64)
    x1 = np.clip(np.floor((mx.astype(f) + r15) * f(0.0625)), 0, gw).astype(np.int64)
    y0 = np.clip(np.floor((my.astype(f) - r32) * f(0.0625)), 0, gh).astype(np.int64)
    y1 = np.clip(np.floor((my.astype(f) + r15) * f(0.0625)), 0, gh).astype(np.int64)
    return x0, x1, y0, y1


def cpu_box_tiles(m, h, g):
    """Tiles [t0, t1) of one axis that the box [m - h, m + h] reaches with a
    pixel (tile t spans pixels 16 t .. 16 t + 15), clamped to [0, g): the
    projection's range, from the same FP32 operations."""
    f32 = np.float32
    m = np.asarray(m, f32)
    h = np.asarray(h, f32)
    lo = (m - h).astype(f32)
    hi = (m + h).astype(f32)
    f = np.floor((lo * f32(0.0625)).astype(f32))
    first = np.where(lo <= (f * f32(16)).astype(f32) + f32(15), f, (f + f32(1)).astype(f32))
    last = (np.floor((hi * f32(0.0625)).astype(f32)) + f32(1)).astype(f32)
    t0 = np.clip(first, 0, g).astype(np.int64)
    t1 = np.clip(last, 0, g).astype(np.int64)
    return t0, t1


def cpu_cut_rect(mx, my, r, hx, hy, W, H):
    """The radius' tile rect cut to the tiles the alpha box reaches (empty:
    x1 <= x0 or y1 <= y0)."""
    gw, gh = (W + 15) // 16, (H + 15) // 16
    x0, x1, y0, y1 = cpu_rect(mx, my, r, W, H)
    bx0, bx1 = cpu_box_tiles(mx, hx, gw)
    by0, by1 = cpu_box_tiles(my, hy, gh)
    return np.maximum(x0, bx0), np.minimum(x1, bx1), np.maximum(y0, by0), np.minimum(y1, by1)


def expected_binning(rec0, rec2, rec3, cams, n, stride):
    """Keys, values and ranges recomputed on the CPU from the GPU's projection
    (vectorised: one entry per (view, Gaussian, tile of the cut rect), stable
    sort by key, so equal keys stay in Gaussian order)."""
    tile_off, t = [], 0
    for c in cams:
        tile_off.append(t)
        t += ((c["width"] + 15) // 16) * ((c["height"] + 15) // 16)
    bins = t
    all_keys, all_vals, per_view = [], [], []
    for v, c in enumerate(cams):
        sl = slice(v * stride, v * stride + n)
        mx, my = rec0[sl, 0], rec0[sl, 1]
        rad = rec3[sl, 0].astype(np.int64)
        tiles = rec3[sl, 1].astype(np.int64)
        x0, x1, y0, y1 = cpu_cut_rect(mx, my, rad, rec2[sl, 1], rec2[sl, 2], c["width"], c["height"])
        w = np.where(tiles > 0, np.maximum(x1 - x0, 0), 0)
        h = np.where(tiles > 0, np.maximum(y1 - y0, 0), 0)
        area = w * h
        per_view.append(int(area.sum()))
        g = np.repeat(np.arange(n, dtype=np.int64), area)
        start = np.repeat(np.cumsum(area) - area, area)
        local = np.arange(area.sum(), dtype=np.int64) - start
        wg = np.maximum(w[g], 1)
        tx = x0[g] + local % wg
        ty = y0[g] + local // wg
        gw = (c["width"] + 15) // 16
        dbits = np.ascontiguousarray(rec2[sl, 3]).view(np.uint32).astype(np.uint64)[g]
        keys = ((tile_off[v] + ty * gw + tx).astype(np.uint64) << np.uint64(32)) | dbits
        all_keys.append(keys)
        all_vals.append(g)
    keys = np.concatenate(all_keys) if all_keys else np.zeros(0, np.uint64)
    vals = np.concatenate(all_vals) if all_vals else np.zeros(0, np.int64)
    # emission order (Gaussian-major across views) does not matter after a
    # stable sort: within a bin (one view) the order is by Gaussian index
    order = np.argsort(keys, kind="stable")
    keys, vals = keys[order], vals[order]
    ranges = np.zeros((bins, 2), dtype=np.int64)
    if keys.size:
        b = (keys >> np.uint64(32)).astype(np.int64)
        starts = np.r_[0, np.nonzero(np.diff(b))[0] + 1]
        ends = np.r_[starts[1:], keys.size]
        ranges[b[starts], 0] = starts
        ranges[b[starts], 1] = ends
    return keys, vals, ranges, np.array(per_view)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
