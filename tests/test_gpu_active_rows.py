"""GPU: the stage layout (active rows in active order): gather / scatter are
exact, and forward, backward and sparse Adam on active rows give what they
give on rows by splat."""
import numpy as np
import pytest
import torch

from paper_2605_13855_gb300 import renderer as R
from paper_2605_13855_gb300 import scenes
from tests.parity_util import to_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("sh_dtype", [torch.float32, torch.bfloat16])
def test_active_rows_match_rows_by_splat(sh_dtype):
    n = 20_000
    scene = scenes.clustered_scene(n, 9500)
    cam = scenes.random_camera(9503, 120, 90)
    mask = scenes.random_active_mask(n, 0.15, 9502)
    sp = R.SplatParams.from_numpy(scene, sh_dtype=sh_dtype)
    r = R.Renderer(n, [(120, 90)])
    r.set_active(torch.as_tensor(mask, device="cuda"))
    r.commit_frozen(sp, cam, 0, mode="recompute")
    act = r.gather_active(sp)
    idx = np.where(mask)[0]
    for k in R.PARAM_NAMES:
        assert torch.equal(getattr(act, k), getattr(sp, k)[torch.as_tensor(idx, device="cuda")]), k
    target = torch.as_tensor(scenes.uniform_target(9504, 120, 90), device="cuda")
    (i1,), l1 = r.forward(sp, [cam], [0], targets=[target])
    g1 = {k: v.clone() for k, v in r.backward(sp).items()}
    (i2,), l2 = r.forward(act, [cam], [0], targets=[target])
    g2 = r.backward(act)
    r.status()
    # the same arithmetic; only the order in which a tile's pairs are summed (the scatter's) differs
    assert (i1 - i2).abs().max().item() <= 4e-6 * i1.abs().max().item()
    assert abs(l1.item() - l2.item()) <= 1e-6 * abs(l1.item())
    for k in g1:  # same arithmetic; float atomics may add in another order
        scale = g1[k].abs().max().item()
        # dL/dsigma is a sum over splats whose terms cancel: its reordering error is relative to
        # the terms, not to the sum, so it gets the gradient bar
        tol = 1e-4 if k == "sigma" else 1e-6
        assert (g1[k] - g2[k]).abs().max().item() <= tol * max(scale, 1e-30), k
    # scatter back after a change of the active rows
    act.means.add_(1.0)
    r.scatter_active(act, sp)
    m = torch.as_tensor(mask.astype(bool), device="cuda")
    assert torch.equal(sp.means[m], act.means)
    assert torch.equal(sp.means[~m].cpu(), torch.as_tensor(scene["means"][~mask.astype(bool)], dtype=torch.float32))
    # the commit needs every splat
    with pytest.raises(R.SparseOITError):
        r.set_active(torch.as_tensor(mask, device="cuda"))
        r.commit_frozen(act, cam, 0, mode="recompute")


def test_adam_on_active_rows_equals_rows_by_splat():
    n = 5000
    rng = np.random.default_rng(3)
    mask = scenes.random_active_mask(n, 0.3, 77)
    r = R.Renderer(n, [(16, 16)])
    r.set_active(torch.as_tensor(mask, device="cuda"))
    idx = torch.as_tensor(np.where(mask)[0], device="cuda")
    na = len(idx)
    full = {k: torch.as_tensor(rng.normal(size=(n,) + R.PARAM_SHAPES[k]), dtype=torch.float32, device="cuda")
            for k in R.PARAM_NAMES}
    m = {k: torch.zeros_like(v) for k, v in full.items()}
    v = {k: torch.zeros_like(t) for k, t in full.items()}
    g = {k: torch.as_tensor(rng.normal(size=(na,) + R.PARAM_SHAPES[k]), dtype=torch.float32, device="cuda")
         for k in R.PARAM_NAMES}
    pa = {k: t[idx].contiguous() for k, t in full.items()}
    ma = {k: t[idx].contiguous() for k, t in m.items()}
    va = {k: t[idx].contiguous() for k, t in v.items()}
    lr = [1e-3] * 8
    for t in (1, 2):
        r.adam_step(g, full, m, v, lr, t)
        r.adam_step(g, pa, ma, va, lr, t)
    torch.cuda.synchronize()
    for k in R.PARAM_NAMES:
        assert torch.equal(full[k][idx], pa[k]) and torch.equal(m[k][idx], ma[k]) and torch.equal(v[k][idx], va[k])
