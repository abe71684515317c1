"""GPU parity on the clustered workload at its stated size: 200,000 splats in 32
anisotropic normal blobs, one 800x800 view, a seeded random 10 % active set
with the frozen complement's sums committed (Sec. 4.1).

* the whole image and every gradient group of the active splats against the
  FP64 oracle (a seeded linear loss, so that no L1 sign decision enters);
* the GPU gradient at 64 parameters sampled uniformly over (active splat,
  parameter field) against FP64 central differences of the oracle's render,
  each difference taken on a window that holds the splat's cutoff ellipse (the
  loss outside it does not change), with h = 1e-6 max(1, |x|).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2605_13855_gb300 import scenes
from paper_2605_13855_gb300.renderer import Renderer, SplatParams
from tests.parity_util import AMB_BAND, AMB_PIX_MAX, GRAD_TOL, IMG_TOL, check_against_oracle, image_error, \
    oracle_grads, to_np

pytestmark = pytest.mark.gpu

PARAMS = ("means", "quats", "log_scales", "opacity_logits", "sh_color", "sh_weight")
WIDTHS = (3, 4, 3, 1, 48, 16)


def _footprint_window(proj_row, W, H, pad=3):
    """Pixel window (x0, y0, x1, y1) that holds the cutoff ellipse {p <= ln(255 o)} of one splat
    (from the oracle's projection row), widened by `pad` pixels."""
    lt = proj_row[22]
    hx, hy = math.sqrt(2.0 * lt * proj_row[3]), math.sqrt(2.0 * lt * proj_row[5])
    x0 = max(0, int(math.floor(proj_row[1] - hx)) - pad)
    x1 = min(W, int(math.ceil(proj_row[1] + hx)) + pad)
    y0 = max(0, int(math.floor(proj_row[2] - hy)) - pad)
    y1 = min(H, int(math.ceil(proj_row[2] + hy)) + pad)
    return x0, y0, x1, y1


def test_clustered_200k_800x800_10pct():
    c = scenes.CLUSTERED
    scene, mask, cam, _ = scenes.clustered_workload()
    n, W, H = c["n"], c["width"], c["height"]
    act = mask.astype(bool)
    rows = np.where(act)[0]
    g = np.random.default_rng(c["seed"] + 7).normal(size=(H, W, 3))

    # FP64 oracle: the complement's sums, the active render over them, the analytic gradient
    famb = np.zeros((3, H, W))
    frozen, _, _ = oracle.render_sums(scene, cam, subset=~act, amb_band=AMB_BAND, amb_sums=famb)
    ref = oracle.render(scene, cam, subset=act, frozen_sums=frozen, amb_band=AMB_BAND, frozen_amb_sums=famb)
    ref_g = oracle_grads(scene, cam, ref["sums"], g, active=act)

    sp = SplatParams.from_numpy(scene)
    r = Renderer(n, [(W, H)])
    r.set_active(torch.as_tensor(mask, device="cuda"))
    r.commit_frozen(sp, cam, 0, mode="recompute")
    images, _ = r.forward(sp, [cam], [0])
    grads = r.backward(sp, [torch.as_tensor(g, dtype=torch.float32, device="cuda")])
    r.status()
    e, frac = image_error(images[0], ref["image"], ref["flip"])
    assert e <= IMG_TOL and frac <= AMB_PIX_MAX, (e, frac)
    errs, excl = check_against_oracle(grads, ref_g, rows)
    print(f"clustered 200k / 800x800 / 10 %: image {e:.2e}, grads {errs}, kink-excluded splats {excl:.2e}")

    # central differences at 64 sampled parameters of active splats away from every threshold
    _, _, amb = oracle.backward(scene, cam, ref["sums"], g, active=act, amb_band=1e-3)
    proj = oracle.project(scene, cam)
    gpu = {k: to_np(grads[k]).reshape(len(rows), -1) for k in PARAMS}
    nz = np.abs(gpu["means"]).max(axis=1) > 0
    cand = np.where((amb[rows] == 0) & (proj[rows, 0] == 1) & nz)[0]
    assert cand.size > 1000
    sc = {k: (v.astype(np.float64).copy() if isinstance(v, np.ndarray) else v) for k, v in scene.items()}
    rng = np.random.default_rng(c["seed"] + 11)
    checked = 0
    for ri in rng.choice(cand, size=64, replace=False):
        i = int(rows[ri])
        gi = int(rng.integers(0, len(PARAMS)))
        name, j = PARAMS[gi], int(rng.integers(0, WIDTHS[gi]))
        win = _footprint_window(proj[i], W, H)
        gw = g[win[1]:win[3], win[0]:win[2]]
        arr = sc[name].reshape(n, -1)
        x0 = arr[i, j]
        h = 1e-6 * max(1.0, abs(x0))
        arr[i, j] = x0 + h
        lp = float(np.sum(oracle.render(sc, cam, window=win)["image"][win[1]:win[3], win[0]:win[2]] * gw))
        arr[i, j] = x0 - h
        lm = float(np.sum(oracle.render(sc, cam, window=win)["image"][win[1]:win[3], win[0]:win[2]] * gw))
        arr[i, j] = x0
        fd = (lp - lm) / (2 * h)
        ga = float(gpu[name][ri, j])
        scale = np.abs(gpu[name]).max()
        assert abs(ga - fd) <= GRAD_TOL * scale + 1e-6 * abs(fd), (name, i, j, ga, fd, scale)
        checked += 1
    assert checked == 64
