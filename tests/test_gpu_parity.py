"""CUDA path against the FP64 oracle, through the C ABI (GPU only).

Tolerances (FP32 path vs FP64 oracle): projection values rel 1e-4 (means in
pixels abs 2e-3), depth bit-exact (both sides evaluate the same FP32
expression), tile counts / keys / values / ranges bit-exact against a CPU
recomputation from the GPU's own FP32 projection, images max-abs 1e-4 and
gradients rel-L2 1e-3 on everything the oracle does not flag as marginal.
"""
import numpy as np
import pytest
import torch

from paper_2509_05216_gb300 import gs, inputs
from tests.gpu_helpers import cpu_cut_rect, expected_binning, rel_l2, run_forward, to_dev_images

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gs.Context(0)
    yield c
    c.close()


def mixed_cams():
    return [inputs.pinhole(inputs.look_at((0.4, -2.8, 1.0)), 200, 152),
            inputs.pinhole(inputs.look_at((2.5, 1.0, -1.2)), 256, 256),
            inputs.pinhole(inputs.look_at((-1.5, 2.0, 1.9)), 97, 131, bg=(0.2, 0.4, 0.1))]


def stack_scene():
    """40 near-isotropic Gaussians stacked along the view axis of the axis
    camera (same screen centre, increasing depth), each with alpha >= 0.6 on
    the centre pixels: without the transmittance stop all 40 would
    contribute there; with it T falls below 1e-4 after about eight."""
    rng = np.random.default_rng(31)
    k = 40
    means = np.stack([rng.uniform(-0.02, 0.02, k), rng.uniform(-0.02, 0.02, k), np.linspace(-0.5, 0.5, k)], 1)
    ls = np.full((k, 3), -1.6) + rng.uniform(-0.1, 0.1, (k, 3))
    q = np.tile([1.0, 0.0, 0.0, 0.0], (k, 1)) + rng.normal(0.0, 0.1, (k, 4))
    o = rng.uniform(0.8, 1.4, k)
    sh = np.zeros((k, 4, 3))
    sh[:, 0, :] = rng.uniform(-1.0, 1.5, (k, 3))
    sh[:, 1:, :] = rng.normal(0.0, 0.3, (k, 3, 3))
    return inputs.pack_params(means, ls, q, o, sh)


def stack_camera():
    return inputs.pinhole(inputs.look_at((0.0, 0.0, 3.0), up=(0.0, 1.0, 0.0)), 64, 48, bg=(0.2, 0.2, 0.5))


SCENES = {
    "sphere_c1": lambda: (inputs.sphere_scene(), [inputs.sphere_camera()]),
    "random_deg3_mixed": lambda: (inputs.random_scene(20000, 3, 11, extent=0.8), mixed_cams()),
    "random_deg1_one": lambda: (inputs.random_scene(5001, 1, 12, extent=0.6, log_scale=(-4, -1.5)),
                                [inputs.pinhole(inputs.look_at((0.1, 0.2, 2.4)), 130, 70)]),
    # strongly anisotropic splats at random angles: the per-warp ellipse cull
    # is tested where the ellipse and its bounding box differ most
    "needles_deg0": lambda: (inputs.random_scene(4000, 0, 13, extent=0.7, log_scale=(-6.0, -1.5)),
                             [inputs.pinhole(inputs.look_at((1.9, -1.6, 1.3)), 192, 160)]),
    # opacity logits 5..8 (opacity 0.9933..0.9997): the 0.99 alpha clamp
    # holds on thousands of (pixel, Gaussian) pairs, and its zero gradient
    # is taken in the backward
    "opaque_deg2": lambda: (inputs.random_scene(3000, 2, 21, extent=0.7, log_scale=(-2.6, -1.6), opacity=(5.0, 8.0)),
                            [inputs.pinhole(inputs.look_at((1.2, -2.2, 1.0)), 160, 128, bg=(0.1, 0.3, 0.2))]),
    # Gaussians far outside the field of view whose splats still reach the
    # image: the slope clamp of J (1.3 half fields of view) is taken by
    # hundreds of visible Gaussians, with its zero derivative
    "guard_band_deg1": lambda: (inputs.random_scene(3000, 1, 22, extent=1.6, log_scale=(-2.0, -0.8),
                                                    opacity=(-1.0, 2.0)),
                                [inputs.pinhole(inputs.look_at((0.3, -2.2, 0.4)), 144, 112)]),
    "stack_deg1": lambda: (stack_scene(), [stack_camera()]),
}


def clamped_alpha_pairs(oracle, scene, cam):
    """(pixel, Gaussian) pairs near each visible mean with opacity G > 0.99."""
    pr = oracle.project(scene, cam)
    count = 0
    for g in np.nonzero((pr["flags"] & oracle.G_VISIBLE) != 0)[0]:
        mx, my = pr["mean2d"][g]
        A, B, C = pr["conic"][g]
        X, Y = np.meshgrid(np.arange(int(mx) - 6, int(mx) + 7), np.arange(int(my) - 6, int(my) + 7))
        inside = (X >= 0) & (X < cam["width"]) & (Y >= 0) & (Y < cam["height"])
        dx, dy = X - mx, Y - my
        G = np.exp(-0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy)
        count += int(((pr["opacity"][g] * G > 0.99) & inside).sum())
    return count


def slope_clamped_visible(oracle, scene, cam):
    """Visible Gaussians whose image-plane slope lies beyond the guard band
    (and not at its edge)."""
    pr = oracle.project(scene, cam)
    P = scene["params"].astype(np.float64)
    n = scene["n"]
    V = np.asarray(cam["viewmat"], np.float64).reshape(4, 4)
    t = V[:3, :3] @ P[0:3, :n] + V[:3, 3:4]
    limx = 1.3 * cam["width"] / (2.0 * cam["fx"])
    limy = 1.3 * cam["height"] / (2.0 * cam["fy"])
    clamped = (np.abs(t[0] / t[2]) > limx) | (np.abs(t[1] / t[2]) > limy)
    ok = ((pr["flags"] & oracle.G_VISIBLE) != 0) & ((pr["flags"] & oracle.G_MARG_GUARD) == 0)
    return int((clamped & ok).sum())


def test_edge_case_scenes_reach_their_branches(oracle):
    """The edge-case scenes do take the branches they are there for."""
    sc, cams = SCENES["opaque_deg2"]()
    assert clamped_alpha_pairs(oracle, sc, cams[0]) > 1000
    sc, cams = SCENES["guard_band_deg1"]()
    assert slope_clamped_visible(oracle, sc, cams[0]) > 200


@pytest.mark.parametrize("name", list(SCENES))
def test_projection_matches_oracle(ctx, oracle, name):
    scene, cams = SCENES[name]()
    run_forward(ctx, scene, cams)
    n, stride = scene["n"], scene["params"].shape[1]
    r0 = ctx.gs_get_buffer(gs.GS_BUF_REC0).cpu().numpy().astype(np.float64)
    r1 = ctx.gs_get_buffer(gs.GS_BUF_REC1).cpu().numpy().astype(np.float64)
    r2f = ctx.gs_get_buffer(gs.GS_BUF_REC2).cpu().numpy()
    r2 = r2f.astype(np.float64)
    r3 = ctx.gs_get_buffer(gs.GS_BUF_REC3).cpu().numpy()
    vm = ctx.gs_get_buffer(gs.GS_BUF_VISMASK).cpu().numpy().view(np.uint64)
    for v, cam in enumerate(cams):
        sl = slice(v * stride, v * stride + n)
        pr = oracle.project(scene, cam)
        vis = (pr["flags"] & oracle.G_VISIBLE) != 0
        touched = ((vm[:n] >> np.uint64(v)) & np.uint64(1)) != 0
        margin = (pr["flags"] & oracle.G_MARG_RECT) != 0
        # visibility (the radius' rect meets the view) and radius agree
        # except on marginal rects
        bad = (touched != vis) & ~margin
        assert not bad.any(), ("visibility differs", np.nonzero(bad)[0][:8], pr["ext"][bad][:8])
        assert np.all(r3[sl, 0][~touched] == 0)
        # instances: the radius' rect cut to the tiles the alpha box reaches,
        # never more than the oracle's rect holds
        x0, x1, y0, y1 = cpu_cut_rect(r0[sl, 0].astype(np.float32), r0[sl, 1].astype(np.float32),
                                      r3[sl, 0].astype(np.int64), r2f[sl, 1], r2f[sl, 2], cam["width"], cam["height"])
        cut = np.where(touched, np.maximum(x1 - x0, 0) * np.maximum(y1 - y0, 0), 0)
        assert np.array_equal(r3[sl, 1].astype(np.int64), cut)
        assert np.all(cut[~margin] <= pr["tiles"][~margin])
        rad = r3[sl, 0]
        both = vis & touched
        # the radius ceil itself may flip where 3 sqrt(lambda) is within FP32
        # reach of an integer (the rect usually does not change then)
        ext = pr["ext"]
        near_int = np.abs(ext - np.round(ext)) <= 1e-5 * ext
        bad = both & ~margin & ~near_int & (rad != pr["radius"])
        assert not bad.any(), ("radius differs", rad[bad][:8], pr["radius"][bad][:8], pr["ext"][bad][:8])
        # depth: the same FP32 evaluation on both sides
        dep = r2f[sl, 3]
        assert np.array_equal(dep[both], pr["depth"][both].astype(np.float32))
        m = both
        L = gs.LOG2E
        conic = np.stack([r0[sl][m, 2] / (-0.5 * L), r0[sl][m, 3] / (-L), r1[sl][m, 0] / (-0.5 * L)], 1)
        np.testing.assert_allclose(r0[sl][m, 0:2], pr["mean2d"][m], rtol=0, atol=2e-3)
        scale = np.abs(pr["conic"][m]).max(axis=1, keepdims=True)
        assert np.all(np.abs(conic - pr["conic"][m]) <= 1e-4 * scale)
        np.testing.assert_allclose(r1[sl][m, 1], pr["opacity"][m], rtol=1e-6, atol=0)
        rgb = np.concatenate([r1[sl][m, 2:4], r2[sl][m, 0:1]], axis=1)
        np.testing.assert_allclose(rgb, pr["rgb"][m], rtol=0, atol=2e-5)
        # the cull box contains the exact alpha >= 1/255 ellipse's box
        A, B, C = pr["conic"][m].T
        det = A * C - B * B
        tau = 2.0 * np.log(np.maximum(255.0 * pr["opacity"][m], 1e-300))
        reach = tau > 0
        hx = np.sqrt(np.where(reach, tau, 0) * C / det)
        hy = np.sqrt(np.where(reach, tau, 0) * A / det)
        assert np.all(r2[sl][m, 1][reach] >= hx[reach])
        assert np.all(r2[sl][m, 2][reach] >= hy[reach])
        assert np.all(r2[sl][m, 1][~reach] < -1e30)


@pytest.mark.parametrize("name", list(SCENES))
def test_binning_is_bit_exact(ctx, name):
    scene, cams = SCENES[name]()
    run_forward(ctx, scene, cams)
    n, stride = scene["n"], scene["params"].shape[1]
    r0 = ctx.gs_get_buffer(gs.GS_BUF_REC0).cpu().numpy()
    r2 = ctx.gs_get_buffer(gs.GS_BUF_REC2).cpu().numpy()
    r3 = ctx.gs_get_buffer(gs.GS_BUF_REC3).cpu().numpy()
    keys, vals, ranges, per_view = expected_binning(r0, r2, r3, cams, n, stride)
    gk = ctx.gs_get_buffer(gs.GS_BUF_KEYS).cpu().numpy().view(np.uint32)
    gv = ctx.gs_get_buffer(gs.GS_BUF_VALS).cpu().numpy().astype(np.int64)
    gr = ctx.gs_get_buffer(gs.GS_BUF_RANGES).cpu().numpy().astype(np.int64)
    inst, bins, _ = ctx.gs_get_counts()
    assert inst == keys.size == per_view.sum()
    # per-(view, Gaussian) tile counts equal the cut rects' areas
    for v in range(len(cams)):
        t = r3[v * stride: v * stride + n, 1].astype(np.int64)
        assert int(t.sum()) == int(per_view[v])
    # the bins of the sorted (bin, depth) keys; within a bin the Gaussians in
    # (depth, index) order
    assert np.array_equal(gk, (keys >> np.uint64(32)).astype(np.uint32))
    assert np.array_equal(gv, vals)
    assert np.array_equal(gr, ranges)
    # the packed (cut) tile rect of every (view, Gaussian) pair with tiles
    for v, c in enumerate(cams):
        sl = slice(v * stride, v * stride + n)
        x0, x1, y0, y1 = cpu_cut_rect(r0[sl, 0], r0[sl, 1], r3[sl, 0].astype(np.int64), r2[sl, 1], r2[sl, 2],
                                      c["width"], c["height"])
        on = r3[sl, 1] > 0
        px, py = r3[sl, 2].astype(np.int64), r3[sl, 3].astype(np.int64)
        assert np.array_equal((px & 0xFFFF)[on], x0[on]) and np.array_equal((px >> 16)[on], x1[on])
        assert np.array_equal((py & 0xFFFF)[on], y0[on]) and np.array_equal((py >> 16)[on], y1[on])
    # both sorts ran only the passes whose digit varies in some view
    ctrl = ctx.gs_get_buffer(gs.GS_BUF_SORT_CTRL).cpu().numpy().astype(np.int64)
    npass = ctrl.size - 1
    # the instances of each view are sorted on bin - view's first bin
    offs = np.cumsum([0] + [((c["width"] + 15) // 16) * ((c["height"] + 15) // 16) for c in cams])
    b = (keys >> np.uint64(32)).astype(np.int64)
    view = np.searchsorted(offs, b, side="right") - 1
    local = b - offs[view]
    assert (1 << (8 * npass)) >= max(offs[1:] - offs[:-1]) > (1 << (8 * (npass - 1)))
    for p in range(npass):
        dg = (local >> (8 * p)) & 255
        one = all(np.unique(dg[view == v]).size <= 1 for v in range(len(cams)))
        assert bool(ctrl[p] & 2) == one
    # the visible Gaussians of each view are sorted on their depth bits
    dctrl = ctx.gs_get_buffer(gs.GS_BUF_DEPTH_CTRL).cpu().numpy().astype(np.int64)
    assert dctrl.size == 5
    dbits = [np.ascontiguousarray(r2[v * stride:v * stride + n, 3]).view(np.uint32)[r3[v * stride:v * stride + n, 1] > 0]
             for v in range(len(cams))]
    for p in range(4):
        one = all(np.unique((d >> (8 * p)) & 255).size <= 1 for d in dbits)
        assert bool(dctrl[p] & 2) == one


def test_binning_with_empty_and_uneven_views(ctx):
    """Views that see nothing (first, middle, last) among views of different
    sizes: the per-view segments of both sorts stay aligned."""
    scene = inputs.random_scene(9000, 2, 14, extent=0.7)
    away = inputs.pinhole(inputs.look_at((0.0, 0.0, 3.0), target=(0.0, 0.0, 6.0), up=(0.0, 1.0, 0.0)), 64, 48)
    cams = [away, mixed_cams()[0], away, mixed_cams()[2], inputs.pinhole(inputs.look_at((2.2, -1.0, 0.4)), 33, 17),
            away]
    run_forward(ctx, scene, cams)
    n, stride = scene["n"], scene["params"].shape[1]
    r0 = ctx.gs_get_buffer(gs.GS_BUF_REC0).cpu().numpy()
    r2 = ctx.gs_get_buffer(gs.GS_BUF_REC2).cpu().numpy()
    r3 = ctx.gs_get_buffer(gs.GS_BUF_REC3).cpu().numpy()
    keys, vals, ranges, per_view = expected_binning(r0, r2, r3, cams, n, stride)
    assert per_view[0] == per_view[2] == per_view[5] == 0 and per_view[1] > 0 and per_view[3] > 0
    gk = ctx.gs_get_buffer(gs.GS_BUF_KEYS).cpu().numpy().view(np.uint32)
    gv = ctx.gs_get_buffer(gs.GS_BUF_VALS).cpu().numpy().astype(np.int64)
    gr = ctx.gs_get_buffer(gs.GS_BUF_RANGES).cpu().numpy().astype(np.int64)
    assert np.array_equal(gk, (keys >> np.uint64(32)).astype(np.uint32))
    assert np.array_equal(gv, vals)
    assert np.array_equal(gr, ranges)


VARIANTS = [1, 2, 4, 8]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("name", list(SCENES))
def test_image_matches_oracle(ctx, oracle, name, variant):
    scene, cams = SCENES[name]()
    ctx.gs_set_option(gs.GS_OPT_RASTER_FWD, variant)
    ctx.gs_set_option(gs.GS_OPT_RASTER_BWD, variant)
    _, img = run_forward(ctx, scene, cams)
    views = gs.split_images(img, cams)
    tf = ctx.gs_get_buffer(gs.GS_BUF_TFINAL).cpu().numpy()
    off = 0
    for v, cam in enumerate(cams):
        ref, reft, marg, _ = oracle.render(scene, cam)
        ok = ~marg
        assert ok.mean() > 0.98
        got = views[v].cpu().numpy()
        assert np.isfinite(got).all()
        assert np.abs(got - ref)[:, ok].max() <= 1e-4
        HW = cam["width"] * cam["height"]
        t = tf[off: off + HW].reshape(cam["height"], cam["width"])
        assert np.abs(t - reft)[ok].max() <= 1e-4
        assert t.min() >= np.float32(1e-4) and t.max() <= 1.0
        off += HW


@pytest.mark.parametrize("fwd,bwd", [(1, 1), (2, 2), (4, 4), (8, 8), (2, 8), (8, 2)])
@pytest.mark.parametrize("name", list(SCENES))
def test_gradient_matches_oracle(ctx, oracle, name, fwd, bwd):
    scene, cams = SCENES[name]()
    ctx.gs_set_option(gs.GS_OPT_RASTER_FWD, fwd)
    ctx.gs_set_option(gs.GS_OPT_RASTER_BWD, bwd)
    p, _ = run_forward(ctx, scene, cams)
    rng = np.random.default_rng(7)
    dimgs = []
    for cam in cams:
        _, _, marg, _ = oracle.render(scene, cam)
        d = rng.normal(size=(3, cam["height"], cam["width"])) * (~marg)
        dimgs.append(d)
    grads = torch.zeros_like(p)
    ctx.gs_raster_bwd(p, scene["n"], scene["deg"], to_dev_images(dimgs), grads)
    ctx.gs_sync()
    ref, ref2d = oracle.render_grad(scene, cams, dimgs, want_2d=True)
    n, stride = scene["n"], scene["params"].shape[1]
    keep = np.ones(n, bool)
    for cam in cams:
        keep &= (oracle.gaussian_flags(scene, cam) & oracle.G_MARG_ANY_GRAD) == 0
    g = grads.cpu().numpy().astype(np.float64)
    assert rel_l2(g[:, :n][:, keep], ref[:, :n][:, keep]) <= 1e-3
    # per-plane check of the larger groups, so no group hides behind another
    # (SH bands 1, 2, 3 each on their own: planes 14-22, 23-37, 38-58)
    P = ref.shape[0]
    for lo, hi in [(0, 3), (3, 6), (6, 10), (10, 11), (11, 14), (14, 23), (23, 38), (38, 59)]:
        if hi > P:
            continue
        r = ref[lo:hi, :n][:, keep]
        if np.linalg.norm(r) > 0:
            assert rel_l2(g[lo:hi, :n][:, keep], r) <= 1e-3, (lo, hi)
    # [B*stride][8] records (mu_x, mu_y, A, B), (C, opacity), -, -, then [B*stride][4] records (r, g, b), -
    flat = ctx.gs_get_buffer(gs.GS_BUF_G2D).cpu().numpy().astype(np.float64)
    bn = flat.size // 12
    g2d = np.concatenate([flat[:8 * bn].reshape(bn, 8)[:, :6], flat[8 * bn:].reshape(bn, 4)[:, :3]], axis=1)
    for v in range(len(cams)):
        got = g2d[v * stride: v * stride + n][keep]
        assert rel_l2(got, ref2d[v][keep]) <= 1e-3


@pytest.mark.parametrize("variant", VARIANTS)
def test_transmittance_stop_fires_on_dense_stack(ctx, oracle, variant):
    """On the centre pixels of the stack every one of the 40 Gaussians has
    alpha >= 0.6, so without the stop all 40 would contribute (n_last = 40);
    with it the last contributor comes far earlier, T_final stays >= 1e-4,
    and one more layer would take it below 1e-4."""
    scene, cams = SCENES["stack_deg1"]()
    cam = cams[0]
    ctx.gs_set_option(gs.GS_OPT_RASTER_FWD, variant)
    run_forward(ctx, scene, cams)
    ctx.gs_set_option(gs.GS_OPT_RASTER_FWD, 2)
    nl = ctx.gs_get_buffer(gs.GS_BUF_NLAST).cpu().numpy().reshape(cam["height"], cam["width"])
    tf = ctx.gs_get_buffer(gs.GS_BUF_TFINAL).cpu().numpy().reshape(cam["height"], cam["width"])
    ranges = ctx.gs_get_buffer(gs.GS_BUF_RANGES).cpu().numpy().astype(np.int64)
    vals = ctx.gs_get_buffer(gs.GS_BUF_VALS).cpu().numpy().astype(np.int64)
    pr = oracle.project(scene, cam)
    A, B, C = pr["conic"].T
    gw = (cam["width"] + 15) // 16
    cx, cy = int(round(cam["cx"])), int(round(cam["cy"]))
    checked = 0
    for y in range(cy - 1, cy + 2):
        for x in range(cx - 1, cx + 2):
            dx, dy = x - pr["mean2d"][:, 0], y - pr["mean2d"][:, 1]
            alpha = pr["opacity"] * np.exp(-0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy)
            if alpha.min() < 0.6:
                continue
            t = (y // 16) * gw + (x // 16)
            length = ranges[t, 1] - ranges[t, 0]
            assert length == 40
            assert 1 <= nl[y, x] <= 20 < length
            # the entry right after the last contributor is the one the stop excluded
            nxt = vals[ranges[t, 0] + nl[y, x]]
            assert tf[y, x] >= np.float32(1e-4)
            assert tf[y, x] * (1.0 - alpha[nxt]) < 1e-4 * (1.0 + 1e-3)
            checked += 1
    assert checked >= 4


def test_pair_stats_count_entries_and_contributions(ctx, oracle):
    """gs_pair_stats: the entries equal the sum of n_last exactly; the
    contributing pairs equal the oracle's count of (pixel, Gaussian)
    contributions up to the pixels where FP32 and FP64 may decide a
    threshold differently."""
    scene, cams = SCENES["random_deg3_mixed"]()
    run_forward(ctx, scene, cams)
    entries, contrib = ctx.gs_pair_stats()
    nl = ctx.gs_get_buffer(gs.GS_BUF_NLAST).cpu().numpy().astype(np.int64)
    assert entries == int(nl.sum())
    ref, marginal = 0, 0
    for cam in cams:
        _, _, marg, pairs = oracle.render(scene, cam)
        ref += pairs
        marginal += int(marg.sum())
    assert 0 < contrib <= entries
    # a marginal pixel can differ by a few contributions
    assert abs(contrib - ref) <= 4 * marginal + 1, (contrib, ref, marginal)
    assert abs(contrib - ref) <= 1e-3 * ref


@pytest.mark.parametrize("variant", [2, 8])
def test_longest_first_tile_order_gives_the_same_results(ctx, variant):
    """GS_OPT_TILE_ORDER = 1 only reorders the tiles the compositing kernels
    take: the image, T_final, n_last, the fused L1 loss and its gradient are
    bit-identical, the backward's gradients equal up to FP32 summation
    order."""
    scene, cams = SCENES["random_deg3_mixed"]()
    _, total = gs.image_offsets(cams)
    rng = np.random.default_rng(23)
    tgt = torch.from_numpy(rng.uniform(0, 1, total).astype(np.float32)).cuda()
    p = torch.from_numpy(scene["params"]).cuda()
    out = []
    for order in (0, 1):
        ctx.gs_set_option(gs.GS_OPT_TILE_ORDER, order)
        ctx.gs_set_option(gs.GS_OPT_RASTER_FWD, variant)
        ctx.gs_set_option(gs.GS_OPT_RASTER_BWD, variant)
        ctx.gs_project(p, scene["n"], scene["deg"], cams)
        ctx.gs_bin_sort()
        img, loss, dimg = torch.empty(total, device="cuda"), torch.zeros(1, device="cuda"), torch.empty(total, device="cuda")
        ctx.gs_raster_fwd_l1(img, tgt, loss, dimg)
        grads = torch.zeros_like(p)
        ctx.gs_raster_bwd(p, scene["n"], scene["deg"], dimg, grads)
        ctx.gs_sync()
        out.append((img, loss, dimg, grads, ctx.gs_get_buffer(gs.GS_BUF_TFINAL), ctx.gs_get_buffer(gs.GS_BUF_NLAST)))
    ctx.gs_set_option(gs.GS_OPT_TILE_ORDER, 0)
    ctx.gs_set_option(gs.GS_OPT_RASTER_FWD, 2)
    ctx.gs_set_option(gs.GS_OPT_RASTER_BWD, 2)
    a, b = out
    for k in (0, 1, 2, 4, 5):
        assert torch.equal(a[k], b[k]), k
    assert (torch.linalg.norm(a[3] - b[3]) / torch.linalg.norm(a[3])).item() <= 1e-5


def test_raster_variants_agree(ctx, oracle):
    scene, cams = SCENES["random_deg3_mixed"]()
    out = {}
    for variant in VARIANTS:
        ctx.gs_set_option(gs.GS_OPT_RASTER_FWD, variant)
        _, img = run_forward(ctx, scene, cams)
        out[variant] = np.concatenate([t.cpu().numpy().reshape(3, -1) for t in gs.split_images(img, cams)], 1)
    # FP32 evaluation order differs between variants: compare away from the
    # oracle's marginal decisions
    ok = np.concatenate([~oracle.render(scene, c)[2].reshape(-1) for c in cams])
    for variant in VARIANTS[1:]:
        assert np.abs(out[variant] - out[VARIANTS[0]])[:, ok].max() <= 1e-5
    ctx.gs_set_option(gs.GS_OPT_RASTER_FWD, 2)


def test_options_reject_bad_values(ctx):
    with pytest.raises(gs.GsError):
        ctx.gs_set_option(gs.GS_OPT_RASTER_FWD, 3)
    with pytest.raises(gs.GsError):
        ctx.gs_set_option(99, 1)
    assert ctx.gs_get_option(gs.GS_OPT_RASTER_FWD) in VARIANTS
    assert ctx.gs_get_option(gs.GS_OPT_RASTER_BWD) in VARIANTS
    with pytest.raises(gs.GsError):
        ctx.gs_set_option(gs.GS_OPT_BWD_DIRECT, 33)
    with pytest.raises(gs.GsError):
        ctx.gs_set_option(gs.GS_OPT_BWD_DIRECT, -1)
    assert 0 <= ctx.gs_get_option(gs.GS_OPT_BWD_DIRECT) <= 32
    with pytest.raises(gs.GsError):
        ctx.gs_set_option(gs.GS_OPT_SORT_ITEMS, 8)
    with pytest.raises(gs.GsError):
        ctx.gs_set_option(gs.GS_OPT_TILE_ORDER, 2)
    assert ctx.gs_get_option(gs.GS_OPT_TILE_ORDER) in (0, 1)
    assert ctx.gs_get_option(gs.GS_OPT_SORT_ITEMS) in (12, 16, 20, 24)


@pytest.mark.parametrize("items", [12, 20, 24])
def test_sort_partition_sizes_give_the_same_binning(ctx, items):
    """Every radix-sort partition size (both sorts) gives the same bins,
    values and ranges (bit-exact against the CPU recomputation)."""
    scene, cams = SCENES["random_deg3_mixed"]()
    ctx.gs_set_option(gs.GS_OPT_SORT_ITEMS, items)
    try:
        run_forward(ctx, scene, cams)
        n, stride = scene["n"], scene["params"].shape[1]
        r0 = ctx.gs_get_buffer(gs.GS_BUF_REC0).cpu().numpy()
        r2 = ctx.gs_get_buffer(gs.GS_BUF_REC2).cpu().numpy()
        r3 = ctx.gs_get_buffer(gs.GS_BUF_REC3).cpu().numpy()
        keys, vals, ranges, _ = expected_binning(r0, r2, r3, cams, n, stride)
        assert np.array_equal(ctx.gs_get_buffer(gs.GS_BUF_KEYS).cpu().numpy().view(np.uint32),
                              (keys >> np.uint64(32)).astype(np.uint32))
        assert np.array_equal(ctx.gs_get_buffer(gs.GS_BUF_VALS).cpu().numpy().astype(np.int64), vals)
        assert np.array_equal(ctx.gs_get_buffer(gs.GS_BUF_RANGES).cpu().numpy().astype(np.int64), ranges)
    finally:
        ctx.gs_set_option(gs.GS_OPT_SORT_ITEMS, 16)


@pytest.mark.parametrize("direct", [0, 3, 32])
@pytest.mark.parametrize("bwd", [2, 8])
def test_gradient_direct_atomics_match_oracle(ctx, oracle, bwd, direct):
    """Backward with the per-lane atomic path never (0), for up to 3
    contributing lanes, and always (32)."""
    scene, cams = SCENES["random_deg3_mixed"]()
    ctx.gs_set_option(gs.GS_OPT_RASTER_FWD, 2)
    ctx.gs_set_option(gs.GS_OPT_RASTER_BWD, bwd)
    ctx.gs_set_option(gs.GS_OPT_BWD_DIRECT, direct)
    p, _ = run_forward(ctx, scene, cams)
    rng = np.random.default_rng(8)
    dimgs = [rng.normal(size=(3, c["height"], c["width"])) * (~oracle.render(scene, c)[2]) for c in cams]
    grads = torch.zeros_like(p)
    ctx.gs_raster_bwd(p, scene["n"], scene["deg"], to_dev_images(dimgs), grads)
    ctx.gs_sync()
    ctx.gs_set_option(gs.GS_OPT_BWD_DIRECT, 2)
    ref = oracle.render_grad(scene, cams, dimgs)
    n = scene["n"]
    keep = np.ones(n, bool)
    for cam in cams:
        keep &= (oracle.gaussian_flags(scene, cam) & oracle.G_MARG_ANY_GRAD) == 0
    g = grads.cpu().numpy().astype(np.float64)
    assert rel_l2(g[:, :n][:, keep], ref[:, :n][:, keep]) <= 1e-3


def test_batched_forward_equals_single_views(ctx):
    scene, cams = SCENES["random_deg3_mixed"]()
    _, img = run_forward(ctx, scene, cams)
    batch = [t.clone() for t in gs.split_images(img, cams)]
    for v, cam in enumerate(cams):
        _, one = run_forward(ctx, scene, [cam])
        assert torch.equal(one.view(3, cam["height"], cam["width"]), batch[v])


def test_all_gaussians_behind_camera_give_background(ctx):
    scene = inputs.random_scene(300, 2, 3, extent=0.3)
    cam = inputs.pinhole(inputs.look_at((0.0, 0.0, 3.0), target=(0.0, 0.0, 6.0)), 40, 33, bg=(0.3, 0.2, 0.1))
    _, img = run_forward(ctx, scene, [cam])
    inst, _, _ = ctx.gs_get_counts()
    assert inst == 0
    out = img.view(3, 33, 40).cpu().numpy()
    for c in range(3):
        assert np.all(out[c] == np.float32(cam["bg"][c]))


def test_single_gaussian_and_large_splat(ctx, oracle):
    # one Gaussian filling most of a ragged 100x77 image
    scene = inputs.pack_params(np.zeros((1, 3)), np.full((1, 3), -0.7), np.array([[1.0, 0.2, 0.1, 0.0]]),
                               np.array([1.5]), np.full((1, 1, 3), 0.4))
    cam = inputs.pinhole(inputs.look_at((0.0, -3.0, 0.5)), 100, 77)
    _, img = run_forward(ctx, scene, [cam])
    ref, _, marg, _ = oracle.render(scene, cam)
    got = img.view(3, 77, 100).cpu().numpy()
    assert np.abs(got - ref)[:, ~marg].max() <= 1e-4


def test_l1_loss_matches_oracle(ctx, oracle):
    rng = np.random.default_rng(3)
    x = rng.uniform(size=100003).astype(np.float32)
    y = rng.uniform(size=100003).astype(np.float32)
    y[::97] = x[::97]  # exact ties: sign(0) = 0
    loss = torch.zeros(1, device="cuda")
    grad = torch.zeros(x.size, device="cuda")
    ctx.gs_l1_loss(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), loss, grad)
    ctx.gs_sync()
    ref, gref = oracle.l1(x, y)
    assert abs(loss.item() - ref) <= 1e-6 * ref
    np.testing.assert_allclose(grad.cpu().numpy(), gref, rtol=1e-6, atol=0)


@pytest.mark.parametrize("variant", [2, 8])
def test_fused_forward_l1_matches_separate_calls(ctx, variant):
    """gs_raster_fwd_l1 writes the same image and dL/dimage as gs_raster_fwd
    followed by gs_l1_loss, and the same loss up to summation order; without
    an image output too."""
    scene, cams = SCENES["random_deg3_mixed"]()
    ctx.gs_set_option(gs.GS_OPT_RASTER_FWD, variant)
    p, img = run_forward(ctx, scene, cams)
    _, total = gs.image_offsets(cams)
    rng = np.random.default_rng(12)
    tgt = torch.from_numpy(rng.uniform(0, 1, total).astype(np.float32)).cuda()
    loss_a, grad_a = torch.zeros(1, device="cuda"), torch.empty(total, device="cuda")
    ctx.gs_l1_loss(img, tgt, loss_a, grad_a)
    img_b, loss_b, grad_b = torch.empty(total, device="cuda"), torch.zeros(1, device="cuda"), torch.empty(total, device="cuda")
    ctx.gs_raster_fwd_l1(img_b, tgt, loss_b, grad_b)
    loss_c, grad_c = torch.zeros(1, device="cuda"), torch.empty(total, device="cuda")
    ctx.gs_raster_fwd_l1(None, tgt, loss_c, grad_c)
    ctx.gs_sync()
    ctx.gs_set_option(gs.GS_OPT_RASTER_FWD, 2)
    assert torch.equal(img, img_b)
    assert torch.equal(grad_a, grad_b) and torch.equal(grad_a, grad_c)
    assert abs(loss_a.item() - loss_b.item()) <= 1e-6 * loss_a.item()
    assert loss_b.item() == loss_c.item()


def test_adam_matches_oracle(ctx, oracle):
    rng = np.random.default_rng(4)
    scene = inputs.random_scene(1003, 3, 2)
    P, stride = scene["params"].shape
    n = scene["n"]
    hp = dict(lr_mean=1.6e-4, lr_scale=5e-3, lr_quat=1e-3, lr_opacity=0.05, lr_sh_dc=2.5e-3,
              lr_sh_rest=2.5e-3 / 20, beta1=0.9, beta2=0.999, eps=1e-15)
    lr_planes = np.array([hp["lr_mean"]] * 3 + [hp["lr_scale"]] * 3 + [hp["lr_quat"]] * 4 + [hp["lr_opacity"]]
                         + [hp["lr_sh_dc"]] * 3 + [hp["lr_sh_rest"]] * (P - 14))
    p = torch.from_numpy(scene["params"]).cuda()
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    p64, m64, v64 = scene["params"].astype(np.float64), np.zeros((P, stride)), np.zeros((P, stride))
    for step in range(1, 4):
        g = rng.normal(size=(P, stride)).astype(np.float32)
        g[:, n:] = 0
        ctx.gs_adam(p, torch.from_numpy(g).cuda(), m, v, n, 3, hp, step)
        oracle.adam(p64, g.astype(np.float64), m64, v64, lr_planes, step)
    ctx.gs_sync()
    np.testing.assert_allclose(p.cpu().numpy(), p64, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(m.cpu().numpy(), m64, rtol=1e-5, atol=1e-7)


def test_visible_only_adam_matches_oracle(ctx, oracle):
    """Visible-only Adam after a narrow-field projection: Gaussians that touch
    no tile in either view keep p, m and v; the others match the oracle's
    Adam step.  The visibility mask equals the oracle's tile counts away from
    marginal rects."""
    rng = np.random.default_rng(14)
    scene = inputs.random_scene(3001, 2, 17, extent=1.5)
    P, stride = scene["params"].shape
    n = scene["n"]
    cams = [inputs.pinhole(inputs.look_at((2.5, 1.0, 0.5), target=(0.8, 0.6, 0.4)), 96, 80, fov_x_deg=25.0),
            inputs.pinhole(inputs.look_at((-0.5, -2.6, 0.9), target=(-0.6, 0.5, -0.5)), 64, 64, fov_x_deg=25.0)]
    p = torch.from_numpy(scene["params"]).cuda()
    ctx.gs_project(p, n, scene["deg"], cams)
    ctx.gs_sync()
    vm = ctx.gs_get_buffer(gs.GS_BUF_VISMASK).cpu().numpy().astype(np.int64)
    vis = (vm != 0).astype(np.uint8)
    ref_vis = oracle.visible_in_batch(scene, cams)
    marg = np.zeros(n, bool)
    for c in cams:
        marg |= (oracle.gaussian_flags(scene, c) & (oracle.G_MARG_RECT | oracle.G_MARG_ZNEAR)) != 0
    assert np.array_equal(vis[~marg], ref_vis[~marg])
    assert 0.1 < vis.mean() < 0.9
    for v, c in enumerate(cams):  # bit v = touches a tile of view v
        t = oracle.project(scene, c)["tiles"] > 0
        assert np.array_equal(((vm >> v) & 1).astype(bool)[~marg], t[~marg])
    hp = dict(lr_mean=1.6e-4, lr_scale=5e-3, lr_quat=1e-3, lr_opacity=0.05, lr_sh_dc=2.5e-3,
              lr_sh_rest=2.5e-3 / 20, beta1=0.9, beta2=0.999, eps=1e-15, visible_only=True)
    lr_planes = np.array([hp["lr_mean"]] * 3 + [hp["lr_scale"]] * 3 + [hp["lr_quat"]] * 4 + [hp["lr_opacity"]]
                         + [hp["lr_sh_dc"]] * 3 + [hp["lr_sh_rest"]] * (P - 14))
    m0 = rng.normal(size=(P, stride)).astype(np.float32) * 1e-3
    v0 = np.abs(rng.normal(size=(P, stride))).astype(np.float32) * 1e-6
    m, v = torch.from_numpy(m0).cuda(), torch.from_numpy(v0).cuda()
    p64, m64, v64 = scene["params"].astype(np.float64), m0.astype(np.float64), v0.astype(np.float64)
    for step in range(1, 4):
        g = rng.normal(size=(P, stride)).astype(np.float32)
        g[:, n:] = 0
        ctx.gs_adam(p, torch.from_numpy(g).cuda(), m, v, n, scene["deg"], hp, step)
        oracle.adam_visible(p64, g.astype(np.float64), m64, v64, lr_planes, step, vis, n=n)
    ctx.gs_sync()
    pg, mg, vg = p.cpu().numpy(), m.cpu().numpy(), v.cpu().numpy()
    hid = vis == 0
    assert np.array_equal(pg[:, :n][:, hid], scene["params"][:, :n][:, hid])
    assert np.array_equal(mg[:, :n][:, hid], m0[:, :n][:, hid]) and np.array_equal(vg[:, :n][:, hid], v0[:, :n][:, hid])
    # three steps of up to lr = 0.05 (opacity) each, every step rounded in
    # FP32 (relative 2^-23 of the parameter and about 1e-6 of the step)
    np.testing.assert_allclose(pg[:, :n], p64[:, :n], rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(mg[:, :n], m64[:, :n], rtol=1e-5, atol=1e-7)


def test_adam_sqrt_batch_lr_scaling(ctx, oracle):
    """The optional sqrt(B) learning-rate scaling of batched training: after a
    3-view projection the step equals plain Adam with the rates times sqrt 3."""
    rng = np.random.default_rng(6)
    scene = inputs.random_scene(777, 1, 3)
    P, stride = scene["params"].shape
    n = scene["n"]
    p = torch.from_numpy(scene["params"]).cuda()
    ctx.gs_project(p, n, 1, mixed_cams())
    hp = dict(lr_mean=1e-3, lr_scale=2e-3, lr_quat=3e-3, lr_opacity=4e-2, lr_sh_dc=5e-3, lr_sh_rest=6e-4,
              sqrt_batch_lr=True)
    lr_planes = np.sqrt(3.0) * np.array([hp["lr_mean"]] * 3 + [hp["lr_scale"]] * 3 + [hp["lr_quat"]] * 4
                                        + [hp["lr_opacity"]] + [hp["lr_sh_dc"]] * 3 + [hp["lr_sh_rest"]] * (P - 14))
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    p64, m64, v64 = scene["params"].astype(np.float64), np.zeros((P, stride)), np.zeros((P, stride))
    for step in (1, 2):
        g = rng.normal(size=(P, stride)).astype(np.float32)
        g[:, n:] = 0
        ctx.gs_adam(p, torch.from_numpy(g).cuda(), m, v, n, 1, hp, step)
        oracle.adam(p64, g.astype(np.float64), m64, v64, lr_planes, step)
    ctx.gs_sync()
    np.testing.assert_allclose(p.cpu().numpy(), p64, rtol=1e-6, atol=1e-7)


def test_invalid_arguments_are_rejected(ctx):
    scene = inputs.random_scene(10, 0, 1)
    p = torch.from_numpy(scene["params"]).cuda()
    bad = inputs.pinhole(inputs.look_at((0, 0, 3.0), up=(0, 1, 0)), 0, 10)
    with pytest.raises(gs.GsError) as e:
        ctx.gs_project(p, scene["n"], 0, [bad])
    assert e.value.status == gs.GS_EINVAL
    fresh = gs.Context(0)
    with pytest.raises(gs.GsError) as e:
        fresh.gs_bin_sort()
    assert e.value.status == gs.GS_ESTATE
    fresh.close()
