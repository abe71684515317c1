"""GPU: every launch option of the renderer (forward pixels per thread,
projection lanes per splat, backward splat order, heaviest-first tile order,
backward organisation, persistent rasters) keeps image and gradient parity with the
FP64 oracle, on a ragged view with a frozen complement."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_13855_gb300 import renderer as R
from paper_2605_13855_gb300 import scenes
from tests.parity_util import AMB_BAND, AMB_PIX_MAX, IMG_TOL, check_against_oracle, image_error, oracle_grads

pytestmark = pytest.mark.gpu

OPTIONS = [
    dict(fwd_pixels_per_thread=1), dict(fwd_pixels_per_thread=2), dict(fwd_pixels_per_thread=4),
    dict(proj_lanes_per_splat=1), dict(proj_lanes_per_splat=2), dict(proj_lanes_per_splat=16),
    dict(bwd_walk=2), dict(raster_tile_order=-1), dict(bwd_parallel=2), dict(raster_persistent=1),
    dict(raster_persistent=1, raster_tile_order=-1, bwd_walk=2),
    dict(fwd_pixels_per_thread=2, proj_lanes_per_splat=1, raster_tile_order=-1, bwd_walk=2),
]


@pytest.fixture(scope="module")
def case():
    n = 30_000
    scene = scenes.clustered_scene(n, 9300)
    cam = scenes.random_camera(9303, 141, 99)  # ragged: neither side a multiple of 16
    mask = scenes.random_active_mask(n, 0.2, 9302)
    act = mask.astype(bool)
    frozen, _, _ = oracle.render_sums(scene, cam, subset=~act)
    ref = oracle.render(scene, cam, subset=act, frozen_sums=frozen, amb_band=AMB_BAND)
    g = np.random.default_rng(9304).normal(size=(99, 141, 3))
    ref_g = oracle_grads(scene, cam, ref["sums"], g, active=act)
    return scene, cam, mask, ref, g, ref_g


@pytest.mark.parametrize("opts", OPTIONS, ids=lambda o: ",".join(f"{k}={v}" for k, v in o.items()))
def test_option_keeps_parity(case, opts):
    scene, cam, mask, ref, g, ref_g = case
    n = len(mask)
    sp = R.SplatParams.from_numpy(scene)
    r = R.Renderer(n, [(cam["width"], cam["height"])], **opts)
    r.set_active(torch.as_tensor(mask, device="cuda"))
    r.commit_frozen(sp, cam, 0, mode="recompute")
    (img,), _ = r.forward(sp, [cam], [0])
    grads = r.backward(sp, [torch.as_tensor(g, dtype=torch.float32, device="cuda")])
    r.status()
    e, frac = image_error(img, ref["image"], ref["flip"])
    assert e <= IMG_TOL and frac <= AMB_PIX_MAX, (e, frac)
    check_against_oracle(grads, ref_g, np.where(mask.astype(bool))[0])


def test_autotuned_options_keep_parity(case):
    """sparseoit_autotune picks the forward strip and persistence, and (with targets) the backward's
    splat order and persistence, among the timed candidates; the step it leaves configured keeps
    parity with the oracle."""
    scene, cam, mask, ref, g, ref_g = case
    n = len(mask)
    sp = R.SplatParams.from_numpy(scene)
    r = R.Renderer(n, [(cam["width"], cam["height"])])
    r.set_active(torch.as_tensor(mask, device="cuda"))
    r.commit_frozen(sp, cam, 0, mode="recompute")
    target = torch.rand((cam["height"], cam["width"], 3), device="cuda")
    tune = r.autotune(sp, [cam], [0], targets=[target], reps=2)
    assert tune["fwd_pixels_per_thread"] in (1, 2, 4) and set(tune["ms"]) == {1, 2, 4}
    assert tune["fwd_persistent"] in (0, 1) and tune["fwd_persistent_ms"] > 0
    assert tune["bwd_walk"] in (1, 2) and tune["bwd_persistent"] in (0, 1)
    assert len(tune["bwd_ms"]) == 4 and all(v > 0 for v in tune["bwd_ms"].values())
    (img,), _ = r.forward(sp, [cam], [0])
    grads = r.backward(sp, [torch.as_tensor(g, dtype=torch.float32, device="cuda")])
    r.status()
    e, frac = image_error(img, ref["image"], ref["flip"])
    assert e <= IMG_TOL and frac <= AMB_PIX_MAX, (e, frac)
    check_against_oracle(grads, ref_g, np.where(mask.astype(bool))[0])
