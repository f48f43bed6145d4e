"""Adaptive density control on the GPU against the oracle (GPU only): the
screen-space statistic accumulated by the backward, and one densification
step (clone, split, prune, moments) on a random set."""
import numpy as np
import pytest
import torch

from oracle import densify as OD
from paper_2509_05216_gb300 import gs, inputs
from tests.gpu_helpers import rel_l2, run_forward, to_dev_images

pytestmark = pytest.mark.gpu


def test_statistic_accumulated_by_the_backward_matches_oracle(oracle):
    scene = inputs.random_scene(6000, 2, 51, extent=0.8)
    cams = [inputs.pinhole(inputs.look_at((0.4, -2.8, 1.0)), 160, 120),
            inputs.pinhole(inputs.look_at((2.5, 1.0, -1.2)), 128, 96)]
    n = scene["n"]
    ctx = gs.Context(0)
    ga = torch.zeros(n, device="cuda")
    ct = torch.zeros(n, device="cuda")
    ctx.gs_set_densify_stats(ga, ct)
    p, _ = run_forward(ctx, scene, cams)
    rng = np.random.default_rng(3)
    dimgs = [rng.normal(size=(3, c["height"], c["width"])) * (~oracle.render(scene, c)[2]) for c in cams]
    grads = torch.zeros_like(p)
    for _ in range(2):  # two backward passes accumulate twice
        ctx.gs_raster_bwd(p, n, scene["deg"], to_dev_images(dimgs), grads)
    ctx.gs_sync()
    ctx.gs_set_densify_stats(None, None)
    _, g2d = oracle.render_grad(scene, cams, dimgs, want_2d=True)
    vis = [oracle.project(scene, c)["tiles"] > 0 for c in cams]
    ref_g, ref_c = OD.ndc_grad_stat([g2d[v] for v in range(len(cams))], cams, vis)
    keep = np.ones(n, bool)
    for c in cams:
        keep &= (oracle.gaussian_flags(scene, c) & (oracle.G_MARG_ANY_GRAD | oracle.G_MARG_RECT)) == 0
    got_g, got_c = ga.cpu().numpy().astype(np.float64), ct.cpu().numpy()
    np.testing.assert_array_equal(got_c[keep], 2 * ref_c[keep])
    assert rel_l2(got_g[keep], 2 * ref_g[keep]) <= 1e-3
    ctx.close()


def densify_inputs(seed):
    rng = np.random.default_rng(seed)
    scene = inputs.random_scene(4099, 3, seed, extent=1.0, log_scale=(-6.0, -3.0), opacity=(-7.0, 3.0))
    n = scene["n"]
    P, stride = scene["params"].shape
    # averages on either side of the threshold, away from it
    avg = np.where(rng.uniform(size=n) < 0.4, rng.uniform(3e-4, 1e-3, n), rng.uniform(0.0, 1e-4, n))
    cnt = rng.integers(0, 5, n).astype(np.float32)
    grad = (avg * cnt).astype(np.float32)
    m = rng.normal(size=(P, stride)).astype(np.float32)
    v = np.abs(rng.normal(size=(P, stride))).astype(np.float32)
    noise = rng.normal(size=(n, 2, 3)).astype(np.float32)
    return scene, m, v, grad, cnt, noise


def test_densify_matches_oracle():
    scene, m, v, grad, cnt, noise = densify_inputs(61)
    n, deg = scene["n"], scene["deg"]
    P = scene["params"].shape[0]
    hp = dict(grad_threshold=2e-4, percent_dense=0.01, scene_extent=3.0, min_opacity=0.005, split_n=2)
    ref_p, ref_m, ref_v, kind = OD.densify(scene["params"][:, :n].astype(np.float64), m[:, :n].astype(np.float64),
                                           v[:, :n].astype(np.float64), grad.astype(np.float64),
                                           cnt.astype(np.float64), noise.astype(np.float64), tau=2e-4,
                                           dense=0.01, extent=3.0, min_opacity=0.005)
    assert min((kind == k).sum() for k in range(4)) > 50  # every decision occurs
    cap = 3 * n + 4
    cap += (-cap) % 4
    outs = [torch.full((P, cap), float("nan"), device="cuda") for _ in range(3)]
    ctx = gs.Context(0)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    nout = ctx.gs_densify(t(scene["params"]), t(m), t(v), n, deg, t(grad), t(cnt), t(noise), hp, *outs)
    ctx.gs_sync()
    assert nout == ref_p.shape[1]
    po, mo, vo = (o[:, :nout].cpu().numpy().astype(np.float64) for o in outs)
    np.testing.assert_allclose(po, ref_p, rtol=1e-6, atol=1e-6)
    np.testing.assert_array_equal(mo, ref_m.astype(np.float32).astype(np.float64))
    np.testing.assert_array_equal(vo, ref_v.astype(np.float32).astype(np.float64))
    # an output stride that is too small: the size is reported, nothing written
    small = [torch.zeros((P, 8), device="cuda") for _ in range(3)]
    with pytest.raises(gs.GsError) as e:
        ctx.gs_densify(t(scene["params"]), t(m), t(v), n, deg, t(grad), t(cnt), t(noise), hp, *small)
    assert e.value.status == gs.GS_ECAPACITY and e.value.n_out == nout
    assert not small[0].any()
    ctx.close()
