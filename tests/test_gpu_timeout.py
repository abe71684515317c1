"""GPU: the bounded device-side wait of the binning scan (failure detection without a fault).

The tile scan of Alg. 2's binning runs as one pass with look-back over partitions of 1024 tiles:
each partition waits for the posts of the partitions before it.  With a partition's post withheld
by the host (sparseoit_inject_scan_stall: a flag that nothing sets), every later partition's wait
runs out after its 0.25 s limit, the kernels after the scan do nothing, and sparseoit_status
reports SPARSEOIT_ERR_TIMEOUT.  No GPU fault is raised and the context stays usable: the next
forward renders the same image as before the injection.
"""
import time

import numpy as np
import pytest
import torch

from paper_2605_13855_gb300 import scenes
from paper_2605_13855_gb300._lib import ERR_TIMEOUT, SparseOITError
from paper_2605_13855_gb300.renderer import Renderer, SplatParams

pytestmark = pytest.mark.gpu


def test_scan_wait_runs_out_and_the_context_recovers():
    n, W, H = 20_000, 1024, 640  # 64 x 40 = 2,560 tiles: three scan partitions
    scene = scenes.clustered_scene(n, 7100)
    cam = scenes.random_camera(7103, W, H)
    mask = scenes.random_active_mask(n, 0.10, 7102)
    sp = SplatParams.from_numpy(scene)
    r = Renderer(n, [(W, H)])
    r.set_active(torch.as_tensor(mask, device="cuda"))
    r.commit_frozen(sp, cam, 0, mode="recompute")
    img0, _ = r.forward(sp, [cam], [0])
    img0 = img0[0].clone()
    r.status()

    r.inject_scan_stall(1)  # partition 1 posts nothing: partition 2 waits for it
    t0 = time.perf_counter()
    r.forward(sp, [cam], [0])
    with pytest.raises(SparseOITError) as ei:
        r.status()
    waited = time.perf_counter() - t0
    assert ei.value.code == ERR_TIMEOUT
    assert 0.2 <= waited < 10.0, waited

    # the context recovers: the same forward again, no injection
    img1, _ = r.forward(sp, [cam], [0])
    r.status()
    scale = float(img0.abs().max())
    # the pair order inside a tile follows the scatter's atomics: FP32 sums agree to rounding
    assert float((img1[0] - img0).abs().max()) <= 4e-6 * scale

    # a partition past the last one withholds nothing
    r.inject_scan_stall(1000)
    img2, _ = r.forward(sp, [cam], [0])
    r.status()
    assert float((img2[0] - img0).abs().max()) <= 4e-6 * scale
