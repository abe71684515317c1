"""GPU: the three backward organisations of the ablation (per splat, per pixel
with warp-reduced atomics, per pixel with per-pair atomics) give the oracle's
gradients at the same bar."""
import numpy as np
import pytest
import torch

from paper_2605_13855_gb300 import renderer as R
from paper_2605_13855_gb300 import scenes
from tests.parity_util import check_against_oracle, oracle_grads
import oracle
from tests.parity_util import AMB_BAND

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_backward_organisations_match_oracle(mode):
    n = 20_000
    scene = scenes.clustered_scene(n, 9100)
    cam = scenes.random_camera(9103, 150, 110)
    mask = scenes.random_active_mask(n, 0.10, 9102)
    act = mask.astype(bool)
    sp = R.SplatParams.from_numpy(scene)
    r = R.Renderer(n, [(150, 110)], bwd_parallel=mode)
    r.set_active(torch.as_tensor(mask, device="cuda"))
    r.commit_frozen(sp, cam, 0, mode="recompute")
    g = np.random.default_rng(9104).normal(size=(110, 150, 3))
    r.forward(sp, [cam], [0])
    grads = r.backward(sp, [torch.as_tensor(g, dtype=torch.float32, device="cuda")])
    r.status()
    ref = oracle.render(scene, cam, amb_band=AMB_BAND)
    check_against_oracle(grads, oracle_grads(scene, cam, ref["sums"], g, active=act), np.where(act)[0])


def test_bad_backward_mode_is_rejected():
    with pytest.raises(R.SparseOITError):
        R.Renderer(100, [(16, 16)], bwd_parallel=4)
