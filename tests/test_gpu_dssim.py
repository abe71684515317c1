"""GPU: the 3DGS photometric loss (1 - lambda) L1 + lambda (1 - SSIM) that the
paper keeps (Sec. 5.1), through sparseoit_loss_l1_dssim, against the FP64
oracle: the loss, dL/dC, and the parameter gradients after the backward."""
import numpy as np
import pytest
import torch

import oracle
from oracle import ssim as osm
from paper_2605_13855_gb300 import renderer as R
from paper_2605_13855_gb300 import scenes
from tests.parity_util import AMB_BAND, AMB_PIX_MAX, IMG_TOL, check_against_oracle, image_error, oracle_grads, \
    to_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("W,H,lam", [(160, 128, 0.2), (77, 45, 0.2), (64, 64, 1.0), (48, 40, 0.0)])
def test_l1_dssim_loss_gradient_and_backward(W, H, lam):
    n = 20_000
    scene = scenes.clustered_scene(n, 8100 + W)
    cam = scenes.random_camera(8103 + W, W, H)
    mask = scenes.random_active_mask(n, 0.10, 8102)
    act = mask.astype(bool)
    sp = R.SplatParams.from_numpy(scene)
    r = R.Renderer(n, [(W, H)])
    r.set_active(torch.as_tensor(mask, device="cuda"))
    r.commit_frozen(sp, cam, 0, mode="recompute")
    ref = oracle.render(scene, cam, amb_band=AMB_BAND)
    tgt = scenes.uniform_target(8104 + W, W, H).astype(np.float64)
    d = ref["image"] - tgt
    tgt = np.where((np.abs(d) < 1e-4) & (d != 0), tgt - 1e-4 * np.sign(d), tgt).astype(np.float32)
    target = torch.as_tensor(tgt, device="cuda")
    gimg = torch.empty((H, W, 3), dtype=torch.float32, device="cuda")
    (img,), _ = r.forward(sp, [cam], [0])
    loss = r.loss_l1_dssim([target], lam, grad_images=[gimg])
    grads = r.backward(sp)
    r.status()
    e, frac = image_error(img, ref["image"], ref["flip"])
    assert e <= IMG_TOL and frac <= AMB_PIX_MAX
    # the loss stage on the same inputs (the library's FP32 image): loss and dL/dC
    x = to_np(img)
    lref = osm.loss_l1_dssim(x, tgt, lam)
    assert abs(loss.item() - lref) <= 1e-5 * abs(lref) + 1e-7, (loss.item(), lref)
    gref = osm.grad_l1_dssim(x, tgt, lam)
    gg = to_np(gimg)
    assert np.abs(gg - gref).max() <= 1e-4 * np.abs(gref).max(), np.abs(gg - gref).max() / np.abs(gref).max()
    # against the oracle's own image the loss differs only through the 1e-5 image error
    assert abs(loss.item() - osm.loss_l1_dssim(ref["image"], tgt, lam)) <= 1e-4 * abs(lref) + 1e-6
    # the parameter gradients of L, back-propagated from that dL/dC
    ref_g = oracle_grads(scene, cam, ref["sums"], gref, active=act)
    check_against_oracle(grads, ref_g, np.where(act)[0])


def test_loss_needs_an_unfused_forward():
    n = 2000
    scene = scenes.clustered_scene(n, 8200)
    cam = scenes.random_camera(8201, 40, 32)
    sp = R.SplatParams.from_numpy(scene)
    r = R.Renderer(n, [(40, 32)])
    r.set_active(torch.ones(n, dtype=torch.uint8, device="cuda"))
    r.commit_frozen(sp, cam, 0)
    target = torch.zeros((32, 40, 3), dtype=torch.float32, device="cuda")
    r.forward(sp, [cam], [0], targets=[target])  # fused L1: the state is already the backward's
    with pytest.raises(R.SparseOITError):
        r.loss_l1_dssim([target])
    r.forward(sp, [cam], [0])
    r.loss_l1_dssim([target])
    with pytest.raises(R.SparseOITError):  # the state was turned into the backward state already
        r.loss_l1_dssim([target])
    r.backward(sp)
    r.status()


def test_l1_dssim_over_a_batch_of_views():
    """Two views of different sizes in one call: the loss is the sum of the per-view losses and the
    gradients the sum of the per-view gradients."""
    n = 15_000
    scene = scenes.clustered_scene(n, 8300)
    cams = [scenes.random_camera(8301, 90, 70), scenes.random_camera(8302, 53, 61)]
    mask = scenes.random_active_mask(n, 0.2, 8303)
    act = mask.astype(bool)
    sp = R.SplatParams.from_numpy(scene)
    r = R.Renderer(n, [(c["width"], c["height"]) for c in cams])
    r.set_active(torch.as_tensor(mask, device="cuda"))
    for v, c in enumerate(cams):
        r.commit_frozen(sp, c, v, mode="recompute")
    tg = []
    refs = []
    for k, c in enumerate(cams):
        ref = oracle.render(scene, c, amb_band=AMB_BAND)
        t = scenes.uniform_target(8310 + k, c["width"], c["height"]).astype(np.float64)
        d = ref["image"] - t
        t = np.where((np.abs(d) < 1e-4) & (d != 0), t - 1e-4 * np.sign(d), t).astype(np.float32)
        tg.append(t)
        refs.append(ref)
    imgs, _ = r.forward(sp, cams, [0, 1])
    loss = r.loss_l1_dssim([torch.as_tensor(t, device="cuda") for t in tg], 0.2)
    grads = r.backward(sp)
    r.status()
    xs = [to_np(im) for im in imgs]
    lref = sum(osm.loss_l1_dssim(x, t, 0.2) for x, t in zip(xs, tg))
    assert abs(loss.item() - lref) <= 1e-5 * abs(lref)
    total = None
    for k, c in enumerate(cams):
        rg = oracle_grads(scene, c, refs[k]["sums"], osm.grad_l1_dssim(xs[k], tg[k], 0.2), active=act)
        if total is None:
            total = rg
        else:
            for key in ("grads", "flip", "dsigma", "dsigma_scale", "dsigma_flip"):
                total[key] = total[key] + rg[key]
            total["amb"] = total["amb"] | rg["amb"]
    check_against_oracle(grads, total, np.where(act)[0])
