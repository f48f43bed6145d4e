"""Captured training step (CUDA graph) against the same step run call by
call, and capacity overflow reporting (GPU only)."""
import numpy as np
import pytest
import torch

from paper_2509_05216_gb300 import gs, inputs

pytestmark = pytest.mark.gpu

HP = dict(lr_mean=1e-3, lr_scale=5e-3, lr_quat=1e-3, lr_opacity=0.05, lr_sh_dc=2.5e-3, lr_sh_rest=1e-4)


def setup():
    ref = inputs.random_scene(12000, 3, 41, extent=0.7)
    cur = inputs.perturb(ref, 42)
    cams = [inputs.pinhole(inputs.look_at((0.4, -2.8, 1.0)), 160, 120),
            inputs.pinhole(inputs.look_at((2.5, 1.0, -1.2)), 128, 128),
            inputs.pinhole(inputs.look_at((-1.5, 2.0, 1.9)), 97, 131)]
    return ref, cur, cams


def render(ctx, scene, cams):
    p = torch.from_numpy(scene["params"]).cuda()
    ctx.gs_project(p, scene["n"], scene["deg"], cams)
    ctx.gs_bin_sort()
    _, total = gs.image_offsets(cams)
    img = torch.empty(total, device="cuda")
    ctx.gs_raster_fwd(img)
    ctx.gs_sync()
    return img


class State:
    def __init__(self, scene):
        self.p = torch.from_numpy(scene["params"]).cuda()
        self.g = torch.zeros_like(self.p)
        self.m = torch.zeros_like(self.p)
        self.v = torch.zeros_like(self.p)


@pytest.mark.parametrize("tile_order", [0, 1])
def test_graph_step_matches_call_by_call(tile_order):
    ref, cur, cams = setup()
    n, deg = cur["n"], cur["deg"]
    plain = gs.Context(0)
    targets = render(plain, ref, cams)
    inst, _, _ = plain.gs_get_counts()
    _, total = gs.image_offsets(cams)
    # call by call
    a = State(cur)
    img_a = torch.empty(total, device="cuda")
    d_a = torch.empty(total, device="cuda")
    loss_a = torch.zeros(1, device="cuda")
    # captured
    b = State(cur)
    img_b = torch.empty(total, device="cuda")
    d_b = torch.empty(total, device="cuda")
    loss_b = torch.zeros(1, device="cuda")
    gctx = gs.Context(0, instance_capacity=2 * inst + 1024)
    gctx.gs_set_option(gs.GS_OPT_TILE_ORDER, tile_order)
    scratch = torch.empty(total, device="cuda")
    gctx.gs_train_graph_capture(b.p, b.g, b.m, b.v, n, deg, HP, cams, scratch, img_b, d_b, loss_b)
    for step in range(1, 4):
        plain.gs_project(a.p, n, deg, cams)
        plain.gs_bin_sort()
        plain.gs_raster_fwd(img_a)
        plain.gs_l1_loss(img_a, targets, loss_a, d_a)
        plain.gs_raster_bwd(a.p, n, deg, d_a, a.g)
        plain.gs_adam(a.p, a.g, a.m, a.v, n, deg, HP, step)
        plain.gs_sync()
        gctx.gs_train_graph_launch(cams, targets, step)
        gctx.gs_sync()
        torch.cuda.synchronize()
        assert abs(loss_a.item() - loss_b.item()) <= 1e-5 * loss_a.item()
        if step == 1:
            assert torch.equal(img_a, img_b)
            rel = (torch.linalg.norm(a.g - b.g) / torch.linalg.norm(a.g)).item()
            assert rel <= 1e-4
    # parameters agree up to gradient-sign flips of near-zero components
    # (one Adam step moves a parameter by about its learning rate)
    diff = (a.p - b.p).abs().max().item()
    assert diff <= 3 * 5e-2
    plain.close()
    gctx.close()


def test_graph_host_targets_match_device_targets():
    """gs_train_graph_launch_host (targets uploaded from pinned host memory on
    the copy stream, loss read back) against device-target replays."""
    ref, cur, cams = setup()
    n, deg = cur["n"], cur["deg"]
    plain = gs.Context(0)
    targets = render(plain, ref, cams)
    inst, _, _ = plain.gs_get_counts()
    _, total = gs.image_offsets(cams)
    host_t = targets.cpu().pin_memory()
    runs = []
    for host in (False, True):
        st = State(cur)
        img, d = torch.empty(total, device="cuda"), torch.empty(total, device="cuda")
        loss = torch.zeros(1, device="cuda")
        g = gs.Context(0, instance_capacity=2 * inst + 1024)
        g.gs_train_graph_capture(st.p, st.g, st.m, st.v, n, deg, HP, cams, targets, img, d, loss)
        losses = []
        for step in range(1, 5):
            if host:
                lh = torch.full((1,), float("nan"), pin_memory=True)
                g.gs_train_graph_launch_host(cams, host_t, step, lh)
                g.gs_sync()
                losses.append(float(lh))
            else:
                g.gs_train_graph_launch(cams, targets, step)
                g.gs_sync()
                losses.append(float(loss.item()))
            if step == 1:
                first_img = img.clone()
        torch.cuda.synchronize()
        runs.append((st, losses, first_img, g))
    (a, la, ia, ga), (b, lb, ib, gb) = runs
    assert torch.equal(ia, ib)
    assert abs(la[0] - lb[0]) <= 1e-6 * la[0]
    for x, y in zip(la, lb):
        assert abs(x - y) <= 1e-4 * x
    assert (a.p - b.p).abs().max().item() <= 4 * 5e-2
    for g in (ga, gb):
        g.close()
    plain.close()


def test_graph_capacity_overflow_is_reported():
    ref, cur, cams = setup()
    n, deg = cur["n"], cur["deg"]
    st = State(cur)
    _, total = gs.image_offsets(cams)
    targets = torch.zeros(total, device="cuda")
    img, d, loss = (torch.empty(total, device="cuda") for _ in range(3))
    gctx = gs.Context(0, instance_capacity=1000)
    with pytest.raises(gs.GsError) as e:
        gctx.gs_train_graph_capture(st.p, st.g, st.m, st.v, n, deg, HP, cams, targets, img, d, loss)
    assert e.value.status == gs.GS_ECAPACITY
    gctx.close()


def test_graph_launch_rejects_other_resolutions():
    ref, cur, cams = setup()
    n, deg = cur["n"], cur["deg"]
    st = State(cur)
    plain = gs.Context(0)
    targets = render(plain, ref, cams)
    inst, _, _ = plain.gs_get_counts()
    _, total = gs.image_offsets(cams)
    img, d, loss = (torch.empty(total, device="cuda") for _ in range(3))
    gctx = gs.Context(0, instance_capacity=2 * inst)
    gctx.gs_train_graph_capture(st.p, st.g, st.m, st.v, n, deg, HP, cams, targets, img, d, loss)
    other = [dict(c) for c in cams]
    other[0]["width"] = 64
    with pytest.raises(gs.GsError):
        gctx.gs_train_graph_launch(other, targets, 1)
    with pytest.raises(gs.GsError):
        gs.Context(0).gs_train_graph_launch(cams, targets, 1)
    plain.close()
    gctx.close()
