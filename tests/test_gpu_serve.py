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


def test_each_result_equals_its_alone_render(oracle):
    scene, p = scene_and_tensor()
    cams = mixed_requests(12, 1)
    srv = gs.Server(p, scene["n"], scene["deg"], slots=2, max_batch_views=5)
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
    scene, p = scene_and_tensor()
    cams = mixed_requests(6, 2)
    # a budget that fits about one request at a time
    per = 20000 * (52 + 72) + 200 * 120 * 32
    srv = gs.Server(p, scene["n"], scene["deg"], slots=3, max_batch_views=8,
                    memory_budget_bytes=int(per * 1.5), output_pool_bytes=0)
    outs = [torch.full((3, c["height"], c["width"]), float("nan"), device="cuda") for c in cams]
    tickets = [srv.gs_serve_submit(c, o) for c, o in zip(cams, outs)]
    for t in tickets:
        st, _ = srv.gs_serve_poll(t, 10_000_000)
        assert st == gs.GS_OK
    torch.cuda.synchronize()
    for c, o in zip(cams, outs):
        assert torch.equal(o, render_alone(scene, p, c))
    srv.close()


def test_server_errors():
    scene, p = scene_and_tensor()
    srv = gs.Server(p, scene["n"], scene["deg"], output_pool_bytes=0)
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
