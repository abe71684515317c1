"""GPU: BF16 SH storage, finite differences through the autograd Function,
and gradient accumulation across backward calls."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_13855_gb300 import scenes
from paper_2605_13855_gb300._lib import ERR_STATE, SparseOITError
from paper_2605_13855_gb300.renderer import Renderer, SparseOITRender, SplatParams
from tests.parity_util import AMB_BAND, AMB_PIX_MAX, GRAD_TOL, IMG_TOL, check_against_oracle, grad_errors, \
    image_error, oracle_grads, to_np

pytestmark = pytest.mark.gpu

PARAMS = ("means", "quats", "log_scales", "opacity_logits", "sh_color", "sh_weight")


def _bf16_rounded(scene):
    """The scene with its SH coefficients rounded to bfloat16 (the values the BF16 path stores)."""
    sc = dict(scene)
    for k in ("sh_color", "sh_weight"):
        sc[k] = torch.as_tensor(scene[k]).to(torch.bfloat16).float().numpy()
    return sc


def test_bf16_sh_against_oracle():
    """BF16-stored SH with FP32 accumulation: parity with the oracle fed the
    same BF16-rounded coefficients at the FP32 bars; the error against the
    unrounded FP32 coefficients is reported."""
    n = 20_000
    scene = scenes.clustered_scene(n, 5100)
    cam = scenes.random_camera(5103, 160, 128)
    mask = scenes.random_active_mask(n, 0.10, 5102)
    sc16 = _bf16_rounded(scene)
    sp = SplatParams.from_numpy(scene, sh_dtype=torch.bfloat16)
    r = Renderer(n, [(cam["width"], cam["height"])])
    r.set_active(torch.as_tensor(mask, device="cuda"))
    r.commit_frozen(sp, cam, 0, mode="recompute")
    g = np.random.default_rng(4).normal(size=(cam["height"], cam["width"], 3))
    img, _ = r.forward(sp, [cam], [0])
    grads = r.backward(sp, [torch.as_tensor(g, dtype=torch.float32, device="cuda")])
    r.status()
    act = mask.astype(bool)
    rows = np.where(act)[0]
    ref16 = oracle.render(sc16, cam, amb_band=AMB_BAND)
    e16, frac = image_error(img[0], ref16["image"], ref16["flip"])
    assert e16 <= IMG_TOL and frac <= AMB_PIX_MAX
    errs16, _ = check_against_oracle(grads, oracle_grads(sc16, cam, ref16["sums"], g, active=act), rows)
    # against the FP32 coefficients: quantisation error of the storage, reported
    ref32 = oracle.render(scene, cam, amb_band=AMB_BAND)
    e32, _ = image_error(img[0], ref32["image"], ref32["flip"])
    r32 = oracle_grads(scene, cam, ref32["sums"], g, active=act)
    errs32 = grad_errors(grads, r32["grads"], rows, (r32["amb"][rows] & 2) == 0, r32["flip"])
    print(f"bf16 SH: vs oracle(bf16 inputs) image {e16:.2e} grads {errs16}; "
          f"vs oracle(fp32 inputs) image {e32:.2e} grads {errs32}")
    assert e32 < 1e-2


def test_autograd_function_against_finite_differences():
    """torch.autograd through SparseOITRender: param.grad at 64 sampled active
    parameters against FP64 central differences of the oracle."""
    n = 20_000
    scene = scenes.clustered_scene(n, 2400)
    cam = scenes.random_camera(2403, 120, 100)
    mask = scenes.random_active_mask(n, 0.10, 2402)
    sp = SplatParams.from_numpy(scene)
    r = Renderer(n, [(cam["width"], cam["height"])])
    r.set_active(torch.as_tensor(mask, device="cuda"))
    r.commit_frozen(sp, cam, 0, mode="recompute")
    params = [getattr(sp, k).clone().requires_grad_(True) for k in PARAMS]
    (img,) = SparseOITRender.apply(r, [cam], [0], sp.sigma, sp.bg, *params)
    g = np.random.default_rng(13).normal(size=(cam["height"], cam["width"], 3))
    (img * torch.as_tensor(g, dtype=torch.float32, device="cuda")).sum().backward()
    grads = {k: to_np(p.grad) for k, p in zip(PARAMS, params)}
    ref = oracle.render(scene, cam, amb_band=1e-3)
    _, _, amb = oracle.backward(scene, cam, ref["sums"], g, active=mask.astype(bool), amb_band=1e-3)
    proj = oracle.project(scene, cam)
    cand = np.where(mask.astype(bool) & (amb == 0) & (proj[:, 0] == 1) & (np.abs(grads["means"]).max(1) > 0))[0]
    sc = {k: (v.astype(np.float64).copy() if isinstance(v, np.ndarray) else v) for k, v in scene.items()}
    rng = np.random.default_rng(1)
    widths = [3, 4, 3, 1, 48, 16]
    checked = 0
    for i in rng.choice(cand, size=min(64, cand.size), replace=False):
        gi = int(rng.integers(0, len(PARAMS)))
        name, j = PARAMS[gi], int(rng.integers(0, widths[gi]))
        arr = sc[name].reshape(n, -1)
        x0 = arr[i, j]
        h = 1e-6 * max(1.0, abs(x0))
        arr[i, j] = x0 + h
        lp = float(np.sum(oracle.render(sc, cam)["image"] * g))
        arr[i, j] = x0 - h
        lm = float(np.sum(oracle.render(sc, cam)["image"] * g))
        arr[i, j] = x0
        fd = (lp - lm) / (2 * h)
        ga = float(grads[name].reshape(n, -1)[i, j])
        scale = np.abs(grads[name].reshape(n, -1)[mask.astype(bool)]).max()
        assert abs(ga - fd) <= GRAD_TOL * scale + 1e-6 * abs(fd), (name, i, j, ga, fd)
        checked += 1
    assert checked >= 48
    # inactive rows receive exactly zero
    assert np.all(grads["means"][~mask.astype(bool)] == 0)


def test_backward_accumulate_sums_calls():
    n = 8000
    scene = scenes.unbounded_scene(n, 6100)
    cams = [scenes.random_camera(6103 + k, 96, 72) for k in range(2)]
    mask = scenes.random_active_mask(n, 0.3, 6102)
    sp = SplatParams.from_numpy(scene)
    r = Renderer(n, [(c["width"], c["height"]) for c in cams])
    r.set_active(torch.as_tensor(mask, device="cuda"))
    for v, c in enumerate(cams):
        r.commit_frozen(sp, c, v, mode="recompute")
    gs = [torch.as_tensor(np.random.default_rng(k).normal(size=(72, 96, 3)), dtype=torch.float32, device="cuda")
          for k in range(2)]
    sep = []
    for v in range(2):
        r.forward(sp, [cams[v]], [v])
        sep.append({k: x.clone() for k, x in r.backward(sp, [gs[v]]).items()})
    r.forward(sp, [cams[0]], [0])
    acc = r.backward(sp, [gs[0]])
    r.forward(sp, [cams[1]], [1])
    r.backward(sp, [gs[1]], out=acc, accumulate=True)
    for k in acc:
        want = sep[0][k] + sep[1][k]
        # float atomics sum in a different order in the two cases: rounding-level differences
        assert (acc[k] - want).abs().max().item() <= 1e-5 * max(1e-30, want.abs().max().item()), k


def test_second_backward_of_one_forward():
    """A backward repeated after one forward with targets (fused L1) zeroes the screen-space sums
    itself (the forward's projection zeroed them for the first) and equals the first and a fresh
    forward + backward; after a forward without targets the first backward consumes the forward's
    planes, and a second one is refused."""
    n = 8000
    scene = scenes.unbounded_scene(n, 6200)
    cam = scenes.random_camera(6203, 96, 72)
    mask = scenes.random_active_mask(n, 0.3, 6202)
    sp = SplatParams.from_numpy(scene)
    r = Renderer(n, [(cam["width"], cam["height"])])
    r.set_active(torch.as_tensor(mask, device="cuda"))
    r.commit_frozen(sp, cam, 0, mode="recompute")
    target = torch.as_tensor(np.random.default_rng(21).uniform(size=(72, 96, 3)), dtype=torch.float32, device="cuda")
    r.forward(sp, [cam], [0], targets=[target])
    first = {k: x.clone() for k, x in r.backward(sp).items()}
    second = {k: x.clone() for k, x in r.backward(sp).items()}
    r.forward(sp, [cam], [0], targets=[target])
    fresh = r.backward(sp)
    for k in second:
        # float atomics sum in a different order in the runs: rounding-level differences
        scale = max(1e-30, fresh[k].abs().max().item())
        assert (second[k] - first[k]).abs().max().item() <= 1e-5 * scale, k
        assert (second[k] - fresh[k]).abs().max().item() <= 1e-5 * scale, k
    g = torch.as_tensor(np.random.default_rng(22).normal(size=(72, 96, 3)), dtype=torch.float32, device="cuda")
    r.forward(sp, [cam], [0])
    r.backward(sp, [g])
    with pytest.raises(SparseOITError) as e:
        r.backward(sp, [g])
    assert e.value.code == ERR_STATE


def test_backward_after_foreign_work_on_the_stream():
    """The backward's kernels are programmatic dependents of the operation before them: with a torch
    kernel and a device-to-host copy enqueued between the forward and the backward on the same
    stream, the gradients equal those of the plain sequence."""
    n = 8000
    scene = scenes.unbounded_scene(n, 6300)
    cam = scenes.random_camera(6303, 96, 72)
    mask = scenes.random_active_mask(n, 0.3, 6302)
    sp = SplatParams.from_numpy(scene)
    r = Renderer(n, [(cam["width"], cam["height"])])
    stream = torch.cuda.Stream()
    target = torch.as_tensor(np.random.default_rng(31).uniform(size=(72, 96, 3)), dtype=torch.float32, device="cuda")
    scratch = torch.zeros(1 << 22, device="cuda")
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        r.set_active(torch.as_tensor(mask, device="cuda"), stream=stream)
        r.commit_frozen(sp, cam, 0, mode="recompute", stream=stream)
        _, loss = r.forward(sp, [cam], [0], targets=[target], stream=stream)
        plain = {k: x.clone() for k, x in r.backward(sp, stream=stream).items()}
        _, loss = r.forward(sp, [cam], [0], targets=[target], stream=stream)
        scratch.mul_(2.0).add_(1.0)                       # a foreign kernel on the stream
        host_loss = loss.to("cpu", non_blocking=True)     # and a copy to host memory
        mixed = r.backward(sp, stream=stream)
    stream.synchronize()
    assert np.isfinite(host_loss.item())
    for k in plain:
        scale = max(1e-30, plain[k].abs().max().item())
        assert (mixed[k] - plain[k]).abs().max().item() <= 1e-5 * scale, k
