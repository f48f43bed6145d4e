"""torch.autograd binding: gradients against the FP64 oracle and against
central finite differences of the CUDA forward (GPU only)."""
import numpy as np
import pytest
import torch

from paper_2509_05216_gb300 import autograd, gs, inputs

pytestmark = pytest.mark.gpu


def cams3():
    return [inputs.pinhole(inputs.look_at((0.4, -2.8, 1.0)), 160, 120),
            inputs.pinhole(inputs.look_at((2.5, 1.0, -1.2)), 128, 128)]


def test_autograd_gradient_matches_oracle(oracle):
    scene = inputs.random_scene(8000, 3, 21, extent=0.7)
    cams = cams3()
    ctx = gs.Context(0)
    p = torch.from_numpy(scene["params"]).cuda().requires_grad_(True)
    img = autograd.rasterize(p, scene["n"], scene["deg"], cams, ctx)
    rng = np.random.default_rng(3)
    ws = []
    for cam in cams:
        _, _, marg, _ = oracle.render(scene, cam)
        ws.append(rng.normal(size=(3, cam["height"], cam["width"])) * (~marg))
    w = torch.cat([torch.from_numpy(x.astype(np.float32)).reshape(-1) for x in ws]).cuda()
    (img * w).sum().backward()
    ref = oracle.render_grad(scene, cams, ws)
    n = scene["n"]
    keep = np.ones(n, bool)
    for cam in cams:
        keep &= (oracle.gaussian_flags(scene, cam) & oracle.G_MARG_ANY_GRAD) == 0
    g = p.grad.cpu().numpy().astype(np.float64)
    err = np.linalg.norm(g[:, :n][:, keep] - ref[:, :n][:, keep]) / np.linalg.norm(ref[:, :n][:, keep])
    assert err <= 1e-3
    ctx.close()


def test_autograd_central_differences_on_sampled_parameters(oracle):
    """FP32 central differences of the CUDA forward on 32 sampled parameters of
    visible, non-marginal Gaussians; the image difference is summed in FP64."""
    scene = inputs.random_scene(3000, 3, 22, extent=0.6, log_scale=(-3.0, -2.0))
    cams = cams3()
    n = scene["n"]
    ctx = gs.Context(0)
    p = torch.from_numpy(scene["params"]).cuda().requires_grad_(True)
    rng = np.random.default_rng(5)
    _, total = gs.image_offsets(cams)
    w = torch.from_numpy(rng.normal(size=total).astype(np.float32)).cuda()
    img = autograd.rasterize(p, n, scene["deg"], cams, ctx)
    (img * w).sum().backward()
    g = p.grad.cpu().numpy()
    ok = np.ones(n, bool)
    for cam in cams:
        f = oracle.gaussian_flags(scene, cam)
        ok &= ((f & oracle.G_VISIBLE) != 0) & ((f & oracle.G_MARG_ANY_GRAD) == 0)
    cand = np.nonzero(ok)[0]
    planes = [0, 1, 2, 3, 5, 6, 8, 10, 11, 13, 20, 40]
    picks = [(planes[i % len(planes)], int(rng.choice(cand))) for i in range(32)]
    w64 = w.double()

    def fd(pl, gi, h):
        base = float(p[pl, gi])
        outs = []
        for sgn in (1.0, -1.0):
            q = p.detach().clone()
            q[pl, gi] = base + sgn * h
            ctx.gs_project(q, n, scene["deg"], cams)
            ctx.gs_bin_sort()
            o = torch.empty(total, device="cuda")
            ctx.gs_raster_fwd(o)
            outs.append(o)
        return float(((outs[0].double() - outs[1].double()) * w64).sum()) / (2 * h)

    errs, kept = [], 0
    with torch.no_grad():
        for pl, gi in picks:
            h = 1e-3 * max(1.0, abs(float(p[pl, gi])))
            f1, f2 = fd(pl, gi, h), fd(pl, gi, h / 2)
            scale = max(abs(f1), abs(f2), 1e-2)
            # the render is piecewise smooth (rect, skip and stop decisions):
            # a step that crosses a jump shows as disagreement between h and h/2
            if abs(f1 - f2) > 0.05 * scale:
                continue
            kept += 1
            an = float(g[pl, gi])
            errs.append(abs(f2 - an) / max(abs(an), abs(f2), 1e-2))
    errs = np.array(errs)
    assert kept >= 24
    assert np.median(errs) <= 1e-2
    assert np.mean(errs <= 5e-2) >= 0.9
    ctx.close()


def test_backward_after_context_reuse_is_refused():
    scene = inputs.random_scene(500, 0, 1, extent=0.5)
    cams = cams3()[:1]
    ctx = gs.Context(0)
    p = torch.from_numpy(scene["params"]).cuda().requires_grad_(True)
    img1 = autograd.rasterize(p, scene["n"], 0, cams, ctx)
    autograd.rasterize(p, scene["n"], 0, cams, ctx)  # reuses the context
    with pytest.raises(RuntimeError):
        img1.sum().backward()
    ctx.close()
