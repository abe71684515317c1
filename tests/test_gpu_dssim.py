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
