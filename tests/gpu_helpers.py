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


def expected_binning(rec0, rec2, rec3, cams, n, stride):
    """Keys, values and ranges recomputed on the CPU from the GPU's projection."""
    B = len(cams)
    keys, vals = [], []
    tile_off = []
    t = 0
    for c in cams:
        tile_off.append(t)
        t += ((c["width"] + 15) // 16) * ((c["height"] + 15) // 16)
    bins = t
    rects = []
    for v, c in enumerate(cams):
        sl = slice(v * stride, v * stride + n)
        mx, my = rec0[sl, 0], rec0[sl, 1]
        rad = rec3[sl, 0].astype(np.int64)
        tiles = rec3[sl, 1].astype(np.int64)
        x0, x1, y0, y1 = cpu_rect(mx, my, rad, c["width"], c["height"])
        area = np.where(tiles > 0, (x1 - x0) * (y1 - y0), 0)
        rects.append((x0, x1, y0, y1, area, np.ascontiguousarray(rec2[sl, 3]).view(np.uint32).astype(np.uint64)))
    # emission order: Gaussian, view, ty, tx
    for g in range(n):
        for v, c in enumerate(cams):
            x0, x1, y0, y1, area, dbits = rects[v]
            if area[g] == 0:
                continue
            gw = (c["width"] + 15) // 16
            for ty in range(y0[g], y1[g]):
                for tx in range(x0[g], x1[g]):
                    keys.append(((tile_off[v] + ty * gw + tx) << 32) | int(dbits[g]))
                    vals.append(g)
    keys = np.array(keys, dtype=np.uint64)
    vals = np.array(vals, dtype=np.int64)
    order = np.argsort(keys, kind="stable")
    keys, vals = keys[order], vals[order]
    ranges = np.zeros((bins, 2), dtype=np.int64)
    if keys.size:
        b = (keys >> np.uint64(32)).astype(np.int64)
        starts = np.r_[0, np.nonzero(np.diff(b))[0] + 1]
        ends = np.r_[starts[1:], keys.size]
        ranges[b[starts], 0] = starts
        ranges[b[starts], 1] = ends
    return keys, vals, ranges, np.array([int(r[4].sum()) for r in rects])


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
