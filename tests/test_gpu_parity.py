"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2605_13855_gb300 import scenes
from paper_2605_13855_gb300._lib import ERR_CAPACITY, ERR_INVALID_ARG, ERR_STATE, SparseOITError
from paper_2605_13855_gb300.renderer import Renderer, SparseOITRender, SplatParams
from tests.parity_util import AMB_BAND, AMB_PIX_MAX, GRAD_TOL, IMG_TOL, check_against_oracle, image_error, \
    oracle_grads, to_np

pytestmark = pytest.mark.gpu


def _renderer_for(scene, cams, mask, mode="recompute", max_pairs=0):
    n = scene["means"].shape[0]
    sp = SplatParams.from_numpy(scene)
    r = Renderer(n, [(c["width"], c["height"]) for c in cams], max_pairs=max_pairs)
    r.set_active(torch.as_tensor(mask, device="cuda"))
    for v, c in enumerate(cams):
        r.commit_frozen(sp, c, v, mode=mode)
    return r, sp


def _linear_g(cam, seed):
    return np.random.default_rng(seed).normal(size=(cam["height"], cam["width"], 3))


def _check_view(r, sp, scene, cam, view, mask, seed, check_grads=True, window=None):
    """Forward + backward (linear loss) of one view against the oracle's full render."""
    g = _linear_g(cam, seed)
    if window is not None:
        x0, y0, x1, y1 = window
        gw = np.zeros_like(g)
        gw[y0:y1, x0:x1] = g[y0:y1, x0:x1]
        g = gw
    images, _ = r.forward(sp, [cam], [view])
    grads = r.backward(sp, [torch.as_tensor(g, dtype=torch.float32, device="cuda")])
    r.status()
    ref = oracle.render(scene, cam, window=window, amb_band=AMB_BAND)
    img = to_np(images[0])
    if window is not None:
        x0, y0, x1, y1 = window
        e, frac = image_error(img[y0:y1, x0:x1], ref["image"][y0:y1, x0:x1], ref["flip"][y0:y1, x0:x1])
    else:
        e, frac = image_error(img, ref["image"], ref["flip"])
    assert e <= IMG_TOL, f"image rel err {e:.3g}"
    assert frac <= AMB_PIX_MAX, f"ambiguous pixel fraction {frac:.3g}"
    if not check_grads:
        return e, None
    act = mask.astype(bool)
    ref_g = oracle_grads(scene, cam, ref["sums"], g, active=act, window=window)
    rows = np.where(act)[0]
    errs, excl = check_against_oracle(grads, ref_g, rows)
    print(f"parity {cam['width']}x{cam['height']}: image {e:.2e} (px with allowance > tol {frac:.2e}), grads",
          {k: f"{v:.2e}" for k, v in errs.items()}, f"kink-excluded splats {excl:.2e}")
    return e, errs


def test_tiny_full_active():
    """4,096 splats, 128x128, all active (the tiny workload)."""
    scene, _, cam = scenes.tiny_workload()
    mask = np.ones(scene["means"].shape[0], np.uint8)
    r, sp = _renderer_for(scene, [cam], mask)
    e, errs = _check_view(r, sp, scene, cam, 0, mask, seed=1)
    print("tiny", e, errs)


def test_tiny_fused_l1():
    """Fused L1 loss (target = render of a second splat set) against the oracle."""
    scene, tscene, cam = scenes.tiny_workload()
    n = scene["means"].shape[0]
    ref = oracle.render(scene, cam, amb_band=AMB_BAND)
    target = oracle.render(tscene, cam)["image"]
    # Where the target is within 1e-4 of the render (but not equal) the sign of
    # C - I is decided by rounding; move those target values 1e-4 away so that
    # FP32 and FP64 take the same L1 sign (exact ties, e.g. empty background
    # in both, stay ties: sign(0) = 0 on both sides).
    d = ref["image"] - target
    near = (np.abs(d) < 1e-4) & (d != 0)
    target = np.where(near, target - 1e-4 * np.sign(d), target).astype(np.float32)
    diff = ref["image"] - target.astype(np.float64)
    assert np.abs(diff)[diff != 0].min() > 5e-5
    mask = np.ones(n, np.uint8)
    r, sp = _renderer_for(scene, [cam], mask)
    tg = torch.as_tensor(target, device="cuda")
    images, loss = r.forward(sp, [cam], [0], targets=[tg])
    grads = r.backward(sp)
    HW = cam["width"] * cam["height"]
    lref = np.abs(diff).mean()
    assert abs(loss.item() - lref) <= 1e-5 * lref
    g = np.sign(diff) / (3 * HW)
    ref_g = oracle_grads(scene, cam, ref["sums"], g)
    check_against_oracle(grads, ref_g, np.arange(n))


@pytest.mark.parametrize("frac", [0.0, 0.1, 1.0])
def test_active_set_equals_full_render(frac):
    """Sec. 4.1: rendering A over the frozen sums of its complement equals the
    full render, and A's gradients are those of the full render."""
    n = 20_000
    scene = scenes.clustered_scene(n, 2100)
    cam = scenes.random_camera(2103, 200, 168)
    mask = scenes.random_active_mask(n, frac, 2102)
    r, sp = _renderer_for(scene, [cam], mask)
    if mask.sum() == 0:
        images, _ = r.forward(sp, [cam], [0])
        ref = oracle.render(scene, cam, amb_band=AMB_BAND)
        e, _ = image_error(images[0], ref["image"], ref["flip"])
        assert e <= IMG_TOL
        return
    _check_view(r, sp, scene, cam, 0, mask, seed=5)


def test_active_indices_are_the_mask_compaction():
    n = 100_003
    m1 = scenes.random_active_mask(n, 0.05, 11)
    r = Renderer(n, [(16, 16)])
    r.set_active(torch.as_tensor(m1, device="cuda"))
    assert np.array_equal(r.active_indices().cpu().numpy(), np.where(m1)[0])
    assert r.n_active == int(m1.sum())
    r.set_active(torch.zeros(n, dtype=torch.uint8, device="cuda"))
    assert r.n_active == 0 and r.active_indices().numel() == 0
    r.set_active(torch.ones(n, dtype=torch.bool, device="cuda"))
    assert r.n_active == n


def test_commit_incremental_equals_recompute():
    n = 20_000
    scene = scenes.clustered_scene(n, 2200)
    cam = scenes.random_camera(2203, 160, 120)
    m1 = scenes.random_active_mask(n, 0.10, 1)
    m2 = scenes.random_active_mask(n, 0.10, 2)
    r, sp = _renderer_for(scene, [cam], m1)
    r.set_active(torch.as_tensor(m2, device="cuda"))
    r.commit_frozen(sp, cam, 0, mode="incremental")
    inc = to_np(r.frozen_sums(0))
    r2, _ = _renderer_for(scene, [cam], m2)
    rec = to_np(r2.frozen_sums(0))
    ab = np.zeros((3, cam["height"], cam["width"]))
    ref, _, _ = oracle.render_sums(scene, cam, subset=~m2.astype(bool), amb_band=AMB_BAND, amb_sums=ab)
    # allowance of the near-cut pairs per plane: sum a w max c (P), sum a w (Q), sum a/(1-a) >= |log(1-a)| (log T)
    allow = [ab[2], ab[2], ab[2], ab[1], ab[0]]
    for k in range(5):
        scale = np.abs(ref[k]).max()
        assert np.max(np.abs(inc[k] - ref[k]) - allow[k]) <= 1e-5 * scale, k
        assert np.max(np.abs(rec[k] - ref[k]) - allow[k]) <= 1e-5 * scale, k
    # and the active render over the incremental sums still matches the full render
    _check_view(r, sp, scene, cam, 0, m2, seed=9)


def test_ragged_views_and_culled_splats():
    """Views whose sizes are not multiples of the tile, splats behind the
    camera or beyond sigma, huge and sub-pixel splats."""
    rng = np.random.default_rng(0)
    n = 3000
    scene = scenes.uniform_cube_scene(n, 77)
    # some splats behind / at the camera, some huge, some tiny and faint
    scene["means"][:50] *= 6.0
    scene["log_scales"][50:80] += 2.5
    scene["log_scales"][80:120] -= 2.0
    scene["opacity_logits"][120:160] = -6.5
    cams = [scenes.random_camera(78, 37, 23), scenes.random_camera(79, 129, 65), scenes.random_camera(80, 16, 16)]
    mask = (rng.uniform(size=n) < 0.6).astype(np.uint8)
    r, sp = _renderer_for(scene, cams, mask)
    for v, c in enumerate(cams):
        _check_view(r, sp, scene, c, v, mask, seed=10 + v)


def test_high_opacity_clamped_pairs():
    """Splats opaque enough that alpha reaches the 0.99 clamp near their
    centres (opacity up to 0.9997), a few among ordinary ones: tiles and warps
    with and without such splats take the rasters' clamping and clamp-free
    paths, both against the oracle."""
    rng = np.random.default_rng(5)
    n = 3000
    scene = scenes.uniform_cube_scene(n, 91)
    hi = rng.choice(n, 60, replace=False)
    scene["opacity_logits"][hi] = rng.uniform(4.0, 8.0, size=hi.size)
    scene["log_scales"][hi] += 2.5  # wide enough that several pixels lie where alpha exceeds 0.99
    cams = [scenes.random_camera(92, 96, 80), scenes.random_camera(93, 53, 37)]
    mask = (rng.uniform(size=n) < 0.7).astype(np.uint8)
    r, sp = _renderer_for(scene, cams, mask)
    clamped = 0
    for v, c in enumerate(cams):
        _check_view(r, sp, scene, c, v, mask, seed=30 + v)
        _, _, stats = oracle.render_sums(scene, c)
        clamped += int(stats[1])
    assert clamped > 0  # some pairs were clamped at 0.99


@pytest.mark.parametrize("strip", [1, 2, 4])
def test_counted_evaluations_match_the_oracle(strip):
    """The counting pass of the forward raster (the E of the benchmark's
    evals/s) counts exactly the active (splat, pixel) pairs inside the view
    whose alpha reaches 1/255, for every strip width, with splats that cover
    whole tiles (the untested list) among ordinary ones."""
    n = 6000
    scene = scenes.clustered_scene(n, 5100)
    scene["log_scales"][:40] += 2.0
    cam = scenes.random_camera(5103, 133, 101)
    mask = scenes.random_active_mask(n, 0.5, 5102)
    sp = SplatParams.from_numpy(scene)
    r = Renderer(n, [(cam["width"], cam["height"])], fwd_pixels_per_thread=strip)
    r.set_active(torch.as_tensor(mask, device="cuda"))
    r.commit_frozen(sp, cam, 0)
    r.set_counting(True)
    r.forward(sp, [cam], [0])
    r.status()
    _, E = r.last_counts()
    _, _, stats = oracle.render_sums(scene, cam, subset=mask.astype(bool))
    # FP32 and FP64 may decide a pair within rounding of the 1/255 cut differently
    assert abs(E - int(stats[0])) <= max(2, 1e-4 * int(stats[0])), (E, int(stats[0]))


def test_set_frozen_restores_a_checkpoint():
    """The frozen sums saved from one context and restored into a fresh one
    (device or host copy) give the same active render as a recompute, and
    the restore is refused before set_active or for a bad view."""
    n = 5000
    scene = scenes.clustered_scene(n, 6100)
    cam = scenes.random_camera(6103, 90, 70)
    mask = scenes.random_active_mask(n, 0.2, 6102)
    r, sp = _renderer_for(scene, [cam], mask)
    saved = r.frozen_sums(0)
    (img_ref,), _ = r.forward(sp, [cam], [0])
    img_ref = to_np(img_ref)
    scale = np.abs(img_ref).max()
    for planes in (saved, saved.cpu()):
        r2 = Renderer(n, [(cam["width"], cam["height"])])
        with pytest.raises(SparseOITError) as ei:
            r2.set_frozen(0, planes)
        assert ei.value.code == ERR_STATE
        r2.set_active(torch.as_tensor(mask, device="cuda"))
        rc = r2.lib.sparseoit_set_frozen(r2._ctx, 1, ctypes.c_void_p(planes.data_ptr()), None)  # no view 1
        assert rc == ERR_INVALID_ARG
        r2.set_frozen(0, planes)
        (img,), _ = r2.forward(sp, [cam], [0])
        r2.status()
        assert np.abs(to_np(img) - img_ref).max() <= 1e-6 * scale
        r2.close()


def test_repeat_runs_agree():
    """Two forward + backward passes over the same inputs agree to rounding
    (only the order of a tile's pairs and of float atomics may differ)."""
    scene, _, cam = scenes.tiny_workload()
    n = scene["means"].shape[0]
    mask = scenes.random_active_mask(n, 0.5, 11)
    r, sp = _renderer_for(scene, [cam], mask)
    g = torch.as_tensor(_linear_g(cam, 12), dtype=torch.float32, device="cuda")
    runs = []
    for _ in range(2):
        (img,), _ = r.forward(sp, [cam], [0])
        grads = r.backward(sp, [g])
        r.status()
        runs.append((to_np(img), {k: to_np(v) for k, v in grads.items()}))
    (i0, g0), (i1, g1) = runs
    assert np.abs(i0 - i1).max() <= 1e-6 * np.abs(i0).max()
    for k in g0:
        scale = max(np.abs(g0[k]).max(), 1e-30)
        assert np.abs(g0[k] - g1[k]).max() <= 1e-5 * scale, k


def test_multiview_batch_equals_single_views():
    n = 8000
    scene = scenes.unbounded_scene(n, 3100)
    cams = [scenes.random_camera(3103 + k, w, h) for k, (w, h) in enumerate([(64, 48), (80, 80), (130, 84)])]
    mask = scenes.random_active_mask(n, 0.3, 3)
    r, sp = _renderer_for(scene, cams, mask)
    gs = [torch.as_tensor(_linear_g(c, 40 + k), dtype=torch.float32, device="cuda") for k, c in enumerate(cams)]
    imgs, _ = r.forward(sp, cams, [0, 1, 2])
    imgs = [to_np(x) for x in imgs]
    gb = r.backward(sp, gs)
    gsum = None
    for k, c in enumerate(cams):
        im1, _ = r.forward(sp, [c], [k])
        assert np.abs(to_np(im1[0]) - imgs[k]).max() <= 1e-6 * max(1e-6, np.abs(imgs[k]).max())
        g1 = r.backward(sp, [gs[k]])
        gsum = {kk: to_np(v) for kk, v in g1.items()} if gsum is None else \
            {kk: gsum[kk] + to_np(v) for kk, v in g1.items()}
    for k in gb:
        scale = max(np.abs(gsum[k]).max(), 1e-30)
        assert np.abs(to_np(gb[k]) - gsum[k]).max() <= 1e-5 * scale, k


def test_permutation_invariance_gpu():
    n = 6000
    scene = scenes.clustered_scene(n, 4100)
    cam = scenes.random_camera(4103, 96, 96)
    perm = np.random.default_rng(1).permutation(n)
    sc2 = {k: (v[perm] if isinstance(v, np.ndarray) and v.ndim >= 1 and v.shape[0] == n else v)
           for k, v in scene.items()}
    mask = np.ones(n, np.uint8)
    r1, sp1 = _renderer_for(scene, [cam], mask)
    r2, sp2 = _renderer_for(sc2, [cam], mask)
    a = to_np(r1.forward(sp1, [cam], [0])[0][0])
    b = to_np(r2.forward(sp2, [cam], [0])[0][0])
    # the pairs of a tile are summed in scatter order (any order is correct, App. A): the two
    # renders differ by FP32 re-association only, a few ulps of the per-pixel sums
    d = np.abs(a - b)
    assert d.max() <= 4e-6 * np.abs(a).max()
    assert d.mean() <= 1e-7 * np.abs(a).max()


def test_state_and_capacity_errors():
    scene, _, cam = scenes.tiny_workload()
    n = scene["means"].shape[0]
    sp = SplatParams.from_numpy(scene)
    r = Renderer(n, [(cam["width"], cam["height"])])
    r.set_active(torch.ones(n, dtype=torch.uint8, device="cuda"))
    with pytest.raises(SparseOITError) as ei:
        r.forward(sp, [cam], [0])          # frozen sums never committed
    assert ei.value.code == ERR_STATE
    with pytest.raises(SparseOITError) as ei:
        r.backward(sp, [torch.zeros(cam["height"], cam["width"], 3, device="cuda")])
    assert ei.value.code == ERR_STATE
    r.commit_frozen(sp, cam, 0)
    r.forward(sp, [cam], [0])
    r.status()
    # a pair arena too small for the view: flagged, and a retry after reserve succeeds
    small = Renderer(n, [(cam["width"], cam["height"])], max_pairs=64)
    small.set_active(torch.ones(n, dtype=torch.uint8, device="cuda"))
    small.commit_frozen(sp, cam, 0)
    small.forward(sp, [cam], [0])
    with pytest.raises(SparseOITError) as ei:
        small.status()
    assert ei.value.code == ERR_CAPACITY
    npairs, _ = small.last_counts()
    small.reserve_pairs(npairs)
    img, _ = small.forward(sp, [cam], [0])
    small.status()
    ref = oracle.render(scene, cam, amb_band=AMB_BAND)
    assert image_error(img[0], ref["image"], ref["flip"])[0] <= IMG_TOL


def test_autograd_function_matches_backward():
    scene, _, cam = scenes.tiny_workload()
    n = scene["means"].shape[0]
    mask = scenes.random_active_mask(n, 0.25, 5)
    r, sp = _renderer_for(scene, [cam], mask)
    params = [getattr(sp, k).clone().requires_grad_(True) for k in
              ("means", "quats", "log_scales", "opacity_logits", "sh_color", "sh_weight")]
    (img,) = SparseOITRender.apply(r, [cam], [0], sp.sigma, sp.bg, *params)
    g = torch.as_tensor(_linear_g(cam, 3), dtype=torch.float32, device="cuda")
    (img * g).sum().backward()
    r.forward(sp, [cam], [0])
    ref = r.backward(sp, [g], rows_by_splat=True)
    for p, k in zip(params, ("means", "quats", "log_scales", "opacity_logits", "sh_color", "sh_weight")):
        scale = ref[k].abs().max().item()
        assert (p.grad - ref[k]).abs().max().item() <= 1e-5 * scale, k
    inactive = torch.as_tensor(mask == 0, device="cuda")
    assert torch.all(params[0].grad[inactive] == 0)


def test_finite_difference_64_params():
    """FP64 central finite differences of the oracle at 64 sampled active
    parameters against the GPU's analytic gradient (clustered scene, 10 %
    active, frozen complement)."""
    n = 20_000
    scene = scenes.clustered_scene(n, 2300)
    cam = scenes.random_camera(2303, 120, 100)
    mask = scenes.random_active_mask(n, 0.10, 2302)
    r, sp = _renderer_for(scene, [cam], mask)
    g = _linear_g(cam, 12)
    r.forward(sp, [cam], [0])
    grads = r.backward(sp, [torch.as_tensor(g, dtype=torch.float32, device="cuda")], rows_by_splat=True)
    ref = oracle.render(scene, cam, amb_band=1e-3)
    _, _, amb = oracle.backward(scene, cam, ref["sums"], g, active=mask.astype(bool), amb_band=1e-3)
    proj = oracle.project(scene, cam)
    # splats that are visible, non-ambiguous and have some gradient
    gm = to_np(grads["means"])
    cand = np.where(mask.astype(bool) & (amb == 0) & (proj[:, 0] == 1) & (np.abs(gm).max(axis=1) > 0))[0]
    rng = np.random.default_rng(0)
    names = ["means", "quats", "log_scales", "opacity_logits", "sh_color", "sh_weight"]
    widths = [3, 4, 3, 1, 48, 16]
    sc = {k: (v.astype(np.float64).copy() if isinstance(v, np.ndarray) else v) for k, v in scene.items()}

    def loss():
        return float(np.sum(oracle.render(sc, cam)["image"] * g))

    checked = 0
    for i in rng.choice(cand, size=min(64, cand.size), replace=False):
        gi = rng.integers(0, len(names))
        name, j = names[gi], int(rng.integers(0, widths[gi]))
        arr = sc[name].reshape(n, -1)
        x0 = arr[i, j]
        h = 1e-6 * max(1.0, abs(x0))
        arr[i, j] = x0 + h
        lp = loss()
        arr[i, j] = x0 - h
        lm = loss()
        arr[i, j] = x0
        fd = (lp - lm) / (2 * h)
        ga = float(to_np(grads[name]).reshape(n, -1)[i, j])
        scale = np.abs(to_np(grads[name]).reshape(n, -1)[mask.astype(bool)]).max()
        assert abs(ga - fd) <= GRAD_TOL * scale + 1e-6 * abs(fd), (name, i, j, ga, fd)
        checked += 1
    assert checked >= 48
