"""sparseoit_set_active_async: the active-set update without a host wait.

The compaction and the copy of the set sizes are only enqueued; the next call
that needs |A| waits for that copy.  The results must be those of the
synchronising sparseoit_set_active, and the oracle's.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_13855_gb300 import scenes
from paper_2605_13855_gb300.renderer import Renderer, SplatParams
from tests.parity_util import AMB_BAND, to_np
from tests.test_gpu_parity import _check_view

pytestmark = pytest.mark.gpu


def test_async_set_active_index_list_and_render():
    n = 20_000
    scene = scenes.clustered_scene(n, 2300)
    cam = scenes.random_camera(2303, 160, 120)
    mask = scenes.random_active_mask(n, 0.10, 5)
    sp = SplatParams.from_numpy(scene)
    r = Renderer(n, [(cam["width"], cam["height"])])
    r.set_active(torch.as_tensor(mask, device="cuda"), asynchronous=True)
    # the count and the ascending index list are the mask's (the first read waits for the copy)
    assert r.n_active == int(mask.sum())
    assert np.array_equal(r.active_indices().cpu().numpy(), np.where(mask)[0].astype(np.int32))
    r.commit_frozen(sp, cam, 0, mode="recompute")
    _check_view(r, sp, scene, cam, 0, mask, seed=21)
    r.close()


def test_async_set_active_twice_then_incremental_commit():
    """Two asynchronous updates in a row with no read in between (the second waits for the
    first's counts itself); the incremental commit of the second equals the oracle's sums."""
    n = 20_000
    scene = scenes.clustered_scene(n, 2400)
    cam = scenes.random_camera(2403, 160, 120)
    m1 = scenes.random_active_mask(n, 0.10, 11)
    m2 = scenes.random_active_mask(n, 0.10, 12)
    m3 = scenes.random_active_mask(n, 0.10, 13)
    sp = SplatParams.from_numpy(scene)
    r = Renderer(n, [(cam["width"], cam["height"])])
    r.set_active(torch.as_tensor(m1, device="cuda"))
    r.commit_frozen(sp, cam, 0, mode="recompute")
    r.set_active(torch.as_tensor(m2, device="cuda"), asynchronous=True)
    r.set_active(torch.as_tensor(m3, device="cuda"), asynchronous=True)
    # the view was committed under m1, two sets ago: the commit recomputes (R-F3)
    r.commit_frozen(sp, cam, 0, mode="incremental")
    got = to_np(r.frozen_sums(0))
    ab = np.zeros((3, cam["height"], cam["width"]))
    ref, _, _ = oracle.render_sums(scene, cam, subset=~m3.astype(bool), amb_band=AMB_BAND, amb_sums=ab)
    allow = [ab[2], ab[2], ab[2], ab[1], ab[0]]
    for k in range(5):
        scale = np.abs(ref[k]).max()
        assert np.max(np.abs(got[k] - ref[k]) - allow[k]) <= 1e-5 * scale, k
    # one more asynchronous step: D+ / D- against m3, applied incrementally
    m4 = scenes.random_active_mask(n, 0.10, 14)
    r.set_active(torch.as_tensor(m4, device="cuda"), asynchronous=True)
    r.commit_frozen(sp, cam, 0, mode="incremental")
    got = to_np(r.frozen_sums(0))
    ab = np.zeros((3, cam["height"], cam["width"]))
    ref, _, _ = oracle.render_sums(scene, cam, subset=~m4.astype(bool), amb_band=AMB_BAND, amb_sums=ab)
    allow = [ab[2], ab[2], ab[2], ab[1], ab[0]]
    for k in range(5):
        scale = np.abs(ref[k]).max()
        assert np.max(np.abs(got[k] - ref[k]) - allow[k]) <= 1e-5 * scale, k
    assert r.n_active == int(m4.sum())
    _check_view(r, sp, scene, cam, 0, m4, seed=22)
    r.close()
