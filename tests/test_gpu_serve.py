"""Continuous-batching render server (GPU only): each result equals the same
request rendered alone, mixed-resolution batches, memory admission, errors."""
import numpy as np
import pytest
import torch

from paper_2509_05216_gb300 import gs, inputs

pytestmark = pytest.mark.gpu


def scene_and_tensor():
    scene = inputs.random_scene(20000, 3, 31, extent=0.8)
    return scene, torch.from_numpy(scene["params"]).cuda()


def mixed_requests(k, seed):
    rng = np.random.default_rng(seed)
    sizes = [(64, 64), (96, 80), (128, 128), (200, 120), (48, 160)]
    out = []
    for i in range(k):
        w, h = sizes[i % len(sizes)]
        out.append(inputs.random_orbit_camera(rng, 3.0, w, h))
    return out


def render_alone(scene, p, cam):
    ctx = gs.Context(0)
    ctx.gs_project(p, scene["n"], scene["deg"], [cam])
    ctx.gs_bin_sort()
    img = torch.empty(3 * cam["width"] * cam["height"], device="cuda")
    ctx.gs_raster_fwd(img)
    ctx.gs_sync()
    ctx.close()
    return img.view(3, cam["height"], cam["width"])


MAX_PX = 200 * 160  # the largest request of mixed_requests is 200 x 120


def slot_fixed_bytes(stride, max_batch_views, max_view_pixels):
    """The per-slot reservation documented with gs_serve_cfg."""
    tiles = max_view_pixels // 128 + 64
    return max_batch_views * (72 * stride + 20 * max_view_pixels + 8 * tiles) + (1 << 20)


def instances_alone(scene, p, cam):
    ctx = gs.Context(0)
    ctx.gs_project(p, scene["n"], scene["deg"], [cam])
    ctx.gs_bin_sort()
    inst = ctx.gs_get_counts()[0]
    ctx.close()
    return inst


def test_each_result_equals_its_alone_render(oracle):
    scene, p = scene_and_tensor()
    cams = mixed_requests(12, 1)
    srv = gs.Server(p, scene["n"], scene["deg"], slots=2, max_batch_views=5, memory_budget_bytes=1 << 30,
                    max_view_pixels=MAX_PX)
    tickets = [srv.gs_serve_submit(c) for c in cams]
    got = []
    for t in tickets:
        st, img = srv.gs_serve_poll(t, 10_000_000)
        assert st == gs.GS_OK
        got.append(img.clone())
        srv.gs_serve_release(t)
    stats = srv.gs_serve_stats()
    assert stats["rendered"] == len(cams) and stats["batches"] >= 3
    for cam, img in zip(cams, got):
        assert torch.equal(img, render_alone(scene, p, cam))
    # and one of them against the oracle
    ref, _, marg, _ = oracle.render(scene, cams[1])
    assert np.abs(got[1].cpu().numpy() - ref)[:, ~marg].max() <= 1e-4
    srv.close()


def test_requests_into_caller_buffers_and_admission_by_memory():
    """A budget whose instance room fits about one view per batch: batches
    are split by the instance estimates, overflowing batches are rendered
    again, and every result still equals its alone render."""
    scene, p = scene_and_tensor()
    cams = mixed_requests(6, 2)
    most = max(instances_alone(scene, p, c) for c in cams)
    slots, views = 3, 8
    room = 65536 + int(1.4 * most)
    budget = slots * (slot_fixed_bytes(p.shape[1], views, MAX_PX) + 26 * room)
    srv = gs.Server(p, scene["n"], scene["deg"], slots=slots, max_batch_views=views,
                    memory_budget_bytes=budget, output_pool_bytes=0, max_view_pixels=MAX_PX)
    outs = [torch.full((3, c["height"], c["width"]), float("nan"), device="cuda") for c in cams]
    tickets = [srv.gs_serve_submit(c, o) for c, o in zip(cams, outs)]
    for t in tickets:
        st, _ = srv.gs_serve_poll(t, 10_000_000)
        assert st == gs.GS_OK
    torch.cuda.synchronize()
    for c, o in zip(cams, outs):
        assert torch.equal(o, render_alone(scene, p, c))
    stats = srv.gs_serve_stats()
    _, retried = srv.gs_serve_timeline()
    assert stats["rendered"] == len(cams)
    # no batch held more than two of these views
    assert stats["batches"] - retried >= len(cams) // 2
    srv.close()


def test_a_request_too_large_for_the_room_fails_with_capacity():
    """A view that alone needs more instances than a slot can hold completes
    with GS_ECAPACITY (after its retries), and the server keeps serving."""
    scene, p = scene_and_tensor()
    big = inputs.pinhole(inputs.look_at((0.3, -2.4, 1.0)), 200, 160)
    small = mixed_requests(1, 5)[0]
    need = instances_alone(scene, p, big)
    room = 140000
    assert need > room > instances_alone(scene, p, small) + 10000
    budget = slot_fixed_bytes(p.shape[1], 1, MAX_PX) + 26 * room
    srv = gs.Server(p, scene["n"], scene["deg"], slots=1, max_batch_views=1, memory_budget_bytes=budget,
                    max_view_pixels=MAX_PX)
    t_big = srv.gs_serve_submit(big)
    st, img = srv.gs_serve_poll(t_big, 10_000_000)
    assert st == gs.GS_ECAPACITY and img is None
    t_small = srv.gs_serve_submit(small)
    st, img = srv.gs_serve_poll(t_small, 10_000_000)
    assert st == gs.GS_OK
    assert torch.equal(img, render_alone(scene, p, small))
    srv.close()


def test_two_batches_are_in_flight_at_once():
    """With two slots the worker launches the next batch while the previous
    one runs: on the device timeline (CUDA events on the slots' streams) some
    batches' intervals overlap."""
    scene = inputs.random_scene(150000, 3, 33, extent=0.8)
    p = torch.from_numpy(scene["params"]).cuda()
    rng = np.random.default_rng(9)
    cams = [inputs.random_orbit_camera(rng, 3.0, 1024, 1024) for _ in range(24)]
    srv = gs.Server(p, scene["n"], scene["deg"], slots=2, max_batch_views=2, memory_budget_bytes=8 << 30,
                    max_view_pixels=1024 * 1024)
    for c in cams[:2]:  # learn the instance counts of this size first
        t = srv.gs_serve_submit(c)
        srv.gs_serve_poll(t, 10_000_000)
        srv.gs_serve_release(t)
    tickets = [srv.gs_serve_submit(c) for c in cams]
    for t in tickets:
        st, _ = srv.gs_serve_poll(t, 10_000_000)
        assert st == gs.GS_OK
        srv.gs_serve_release(t)
    spans, _ = srv.gs_serve_timeline()
    assert len(spans) >= 12
    assert all(b > a for a, b in spans)
    overlaps = sum(1 for i in range(len(spans)) for j in range(i + 1, len(spans))
                   if spans[i][0] < spans[j][1] and spans[j][0] < spans[i][1])
    assert overlaps >= 1, spans
    srv.close()


def test_server_errors():
    scene, p = scene_and_tensor()
    with pytest.raises(gs.GsError):  # no room for tile instances in this budget
        gs.Server(p, scene["n"], scene["deg"], memory_budget_bytes=1 << 20, max_view_pixels=MAX_PX)
    srv = gs.Server(p, scene["n"], scene["deg"], output_pool_bytes=0, memory_budget_bytes=1 << 30,
                    max_view_pixels=MAX_PX)
    big = dict(mixed_requests(1, 3)[0])
    big["width"], big["height"] = 400, 100  # 40,000 pixels > MAX_PX
    with pytest.raises(gs.GsError) as e:
        srv.gs_serve_submit(big, torch.empty(3 * 400 * 100, device="cuda"))
    assert e.value.status == gs.GS_EINVAL
    cam = mixed_requests(1, 3)[0]
    with pytest.raises(gs.GsError) as e:
        srv.gs_serve_submit(cam)  # no pool and no output buffer
    assert e.value.status == gs.GS_EINVAL
    with pytest.raises(gs.GsError):
        srv.gs_serve_poll(12345, 0)
    bad = dict(cam)
    bad["width"] = 0
    with pytest.raises(gs.GsError):
        srv.gs_serve_submit(bad, torch.empty(3, device="cuda"))
    srv.close()
