"""GPU: the periodic active-set update (Sec. 4.1, Eq. 8) through the C ABI
against the FP64 oracle: the subsampled views, the gradients summed over
them, the per-group norms and the new mask."""
import numpy as np
import pytest
import torch

import oracle
from oracle import active_set as oas
from paper_2605_13855_gb300 import renderer as R
from paper_2605_13855_gb300 import scenes
from tests.parity_util import AMB_BAND, GRAD_TOL, check_against_oracle, oracle_grads, to_np

pytestmark = pytest.mark.gpu


def _targets_away_from_render(scene, cams, seed):
    """Uniform targets, moved 1e-4 away from the oracle's render where closer (both sides take the same L1 sign)."""
    out, refs = [], []
    for k, cm in enumerate(cams):
        t = scenes.uniform_target(seed + k, cm["width"], cm["height"]).astype(np.float64)
        ref = oracle.render(scene, cm, amb_band=AMB_BAND)
        d = ref["image"] - t
        t = np.where((np.abs(d) < 1e-4) & (d != 0), t - 1e-4 * np.sign(d), t)
        out.append(t.astype(np.float32))
        refs.append(ref)
    return out, refs


def test_activeness_kernel_matches_oracle_norms():
    rng = np.random.default_rng(5)
    n = 5000
    g = rng.normal(size=(n, 75)) * rng.exponential(size=(n, 1))
    g[::7] = 0.0
    eps = np.quantile(oas.group_norms(g), 0.8, axis=0)
    gd = {name: torch.as_tensor(g[:, a:b].reshape((n,) + R.PARAM_SHAPES[name]), dtype=torch.float32, device="cuda")
          .contiguous() for name, (a, b) in zip(R.PARAM_NAMES, oas.GROUP_COLUMNS)}
    mask, norms = R.activeness(gd, eps, with_norms=True)
    gf = np.concatenate([to_np(gd[name]).reshape(n, -1) for name in R.PARAM_NAMES], axis=1)  # the FP32 inputs
    ref_n = oas.group_norms(gf)
    assert np.abs(to_np(norms) - ref_n).max() <= 1e-6 * ref_n.max()
    ref_m = oas.activeness(gf, eps)
    near = (np.abs(ref_n / eps[None, :] - 1.0) < 1e-6).any(axis=1)
    assert np.array_equal(to_np(mask).astype(np.uint8)[~near], ref_m[~near])
    assert near.mean() < 1e-3


def test_update_active_set_matches_oracle():
    n = 20_000
    scene = scenes.clustered_scene(n, 7100)
    cams = [scenes.random_camera(7200 + k, 96, 72) for k in range(6)]
    n_sub, first = 3, 4
    sel_ref = oas.fps_views(cams, n_sub, first)
    targets, refs = _targets_away_from_render(scene, cams, 7300)
    # oracle: sum over the picked views of the full-set L1 gradient (mean over 3HW per view)
    total = None
    for j in sel_ref:
        cm = cams[j]
        W, H = cm["width"], cm["height"]
        gimg = np.sign(refs[j]["image"] - targets[j].astype(np.float64)) / (3.0 * W * H)
        rg = oracle_grads(scene, cm, refs[j]["sums"], gimg, active=np.ones(n, bool))
        if total is None:
            total = rg
        else:
            for k in ("grads", "flip", "dsigma", "dsigma_scale", "dsigma_flip"):
                total[k] = total[k] + rg[k]
            total["amb"] = total["amb"] | rg["amb"]
    norms_ref = oas.group_norms(total["grads"])
    eps = np.quantile(norms_ref[norms_ref.max(axis=1) > 0], 0.9, axis=0)

    sp = R.SplatParams.from_numpy(scene)
    r = R.Renderer(n, [(cm["width"], cm["height"]) for cm in cams])
    prev = scenes.random_active_mask(n, 0.3, 7400)  # a previous active set, view 0 committed under it
    r.set_active(torch.as_tensor(prev, device="cuda"))
    r.commit_frozen(sp, cams[0], 0, mode="recompute")
    tg = [torch.as_tensor(t, device="cuda") for t in targets]
    mask, sel, grads = r.update_active_set(sp, cams, tg, eps, n_sub, first)
    r.status()
    assert sel == sel_ref
    # the summed gradients at the 1e-4 bar (full rows: every splat was active during the update)
    check_against_oracle(grads, total, np.arange(n))
    # the mask is decided by the library's FP32 norms: it must equal the test applied to them
    m = to_np(mask).astype(np.uint8)
    m2, norms = R.activeness(grads, eps, with_norms=True)
    gn = to_np(norms)
    assert np.array_equal(to_np(m2).astype(np.uint8), m)
    assert np.array_equal(m, (gn > np.asarray(eps, np.float32)[None, :]).any(axis=1).astype(np.uint8))
    # those norms against the oracle's: within what the 1e-4 gradient bar and the allowances imply
    # (a group norm moves at most by the norm of its elements' errors, sqrt(48) x the element bar)
    err = np.abs(gn - norms_ref)
    bound = 7 * GRAD_TOL * np.array([np.abs(total["grads"][:, a:b]).max() for a, b in oas.GROUP_COLUMNS])[None, :] \
        + oas.group_norms(total["flip"])
    kink = (total["amb"] & 2) != 0
    assert np.all(err[~kink] <= bound[~kink])
    # and the oracle's mask wherever its margin to a threshold exceeds the library's measured norm error
    ref_m = oas.activeness(total["grads"], eps)
    decided = ~((np.abs(norms_ref - eps[None, :]) <= err).any(axis=1) | kink)
    assert np.array_equal(m[decided], ref_m[decided]), int((m[decided] != ref_m[decided]).sum())
    assert decided.mean() > 0.99, decided.mean()
    assert 0 < ref_m.sum() < n
    # the context now holds the new active set, every view stale until committed
    assert r.n_active == int(m.sum())
    assert torch.equal(r.active_indices().cpu(), torch.as_tensor(np.where(m)[0], dtype=torch.int32))
    with pytest.raises(R.SparseOITError):
        r.forward(sp, [cams[0]], [0])
    # the update left view 0's frozen sums as they were: the incremental commit (+D+ -D- against the
    # previous set) gives the new complement's sums, equal to a recompute and to the oracle
    r.commit_frozen(sp, cams[0], 0, mode="incremental")
    inc = to_np(r.frozen_sums(0))
    ab = np.zeros((3, cams[0]["height"], cams[0]["width"]))
    fz_ref, _, _ = oracle.render_sums(scene, cams[0], subset=~m.astype(bool), amb_band=AMB_BAND, amb_sums=ab)
    # allowance of the near-cut pairs per plane: sum a w max c (P), sum a w (Q), sum a/(1-a) (log T)
    allow = [ab[2], ab[2], ab[2], ab[1], ab[0]]
    for k in range(5):
        assert np.max(np.abs(inc[k] - fz_ref[k]) - allow[k]) <= 1e-5 * np.abs(fz_ref[k]).max(), k
    r.forward(sp, [cams[0]], [0])
    r.status()
