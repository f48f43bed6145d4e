"""SSIM / PSNR metrics and the D-SSIM training loss against the FP64 oracle
(GPU only), on a batch of three views of different sizes (ragged tiles at
every border): per-view SSIM and PSNR, the loss, and its gradient."""
import numpy as np
import pytest
import torch

from oracle import ssim as S
from paper_2509_05216_gb300 import gs, inputs
from tests.gpu_helpers import rel_l2, run_forward

pytestmark = pytest.mark.gpu


def batch():
    scene = inputs.random_scene(20000, 3, 11, extent=0.8)
    cams = [inputs.pinhole(inputs.look_at((0.4, -2.8, 1.0)), 200, 152),
            inputs.pinhole(inputs.look_at((2.5, 1.0, -1.2)), 97, 131),
            inputs.pinhole(inputs.look_at((-1.5, 2.0, 1.9)), 64, 48)]
    return scene, cams


def targets_for(img, seed):
    rng = np.random.default_rng(seed)
    t = img.cpu().numpy() + rng.normal(0.0, 0.05, size=img.numel()).astype(np.float32)
    return torch.from_numpy(np.clip(t, 0.0, 1.0).astype(np.float32)).cuda()


def test_metrics_match_oracle():
    ctx = gs.Context(0)
    scene, cams = batch()
    _, img = run_forward(ctx, scene, cams)
    tgt = targets_for(img, 1)
    ssim, psnr = ctx.gs_image_metrics(img, tgt, len(cams))
    xs, ys = gs.split_images(img, cams), gs.split_images(tgt, cams)
    for v in range(len(cams)):
        x, y = xs[v].cpu().numpy(), ys[v].cpu().numpy()
        assert abs(ssim[v] - S.ssim(x, y)) <= 2e-5
        assert abs(psnr[v] - S.psnr(x, y)) <= 1e-4
    # identical images: SSIM 1
    s1, _ = ctx.gs_image_metrics(img, img, len(cams))
    assert all(abs(s - 1.0) <= 1e-5 for s in s1)
    ctx.close()


@pytest.mark.parametrize("lam", [0.2, 1.0])
def test_dssim_loss_and_gradient_match_oracle(lam):
    ctx = gs.Context(0)
    scene, cams = batch()
    _, img = run_forward(ctx, scene, cams)
    tgt = targets_for(img, 2)
    loss = torch.zeros(1, device="cuda")
    grad = torch.full_like(img, float("nan"))
    ctx.gs_ssim_loss(img, tgt, lam, loss, grad)
    ctx.gs_sync()
    xs = [v.cpu().numpy() for v in gs.split_images(img, cams)]
    ys = [v.cpu().numpy() for v in gs.split_images(tgt, cams)]
    ref_loss, ref_grads = S.dssim_loss(xs, ys, lam)
    assert abs(loss.item() - ref_loss) <= 1e-6 * max(1.0, abs(ref_loss))
    got = [g.cpu().numpy().astype(np.float64) for g in gs.split_images(grad, cams)]
    for g, r in zip(got, ref_grads):
        assert np.isfinite(g).all()
        assert rel_l2(g, r) <= 1e-3
    # the loss alone, and the same gradient again
    loss2, grad2 = torch.zeros(1, device="cuda"), torch.empty_like(img)
    ctx.gs_ssim_loss(img, tgt, lam, loss2, None)
    ctx.gs_ssim_loss(img, tgt, lam, None, grad2)
    ctx.gs_sync()
    assert loss2.item() == loss.item() and torch.equal(grad2, grad)
    ctx.close()


def test_ssim_rejects_bad_arguments():
    ctx = gs.Context(0)
    img = torch.zeros(3 * 8 * 8, device="cuda")
    with pytest.raises(gs.GsError) as e:
        ctx.gs_ssim_loss(img, img, 0.2, torch.zeros(1, device="cuda"), None)
    assert e.value.status == gs.GS_ESTATE
    scene, cams = batch()
    run_forward(ctx, scene, cams[2:])
    img = torch.zeros(3 * 64 * 48, device="cuda")
    with pytest.raises(gs.GsError) as e:
        ctx.gs_ssim_loss(img, img, 1.5, torch.zeros(1, device="cuda"), None)
    assert e.value.status == gs.GS_EINVAL
    ctx.close()
