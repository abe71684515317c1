"""GPU: sparse Adam over the active set (sparseoit_adam_step) against the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import adam as oad
from paper_2605_13855_gb300 import renderer as R
from paper_2605_13855_gb300 import scenes
from tests.parity_util import to_np

pytestmark = pytest.mark.gpu

COLS = dict(means=(0, 3), quats=(3, 7), log_scales=(7, 10), opacity_logits=(10, 11), sh_color=(11, 59),
            sh_weight=(59, 75))


def _split(a, n):
    return {k: torch.as_tensor(a[:, lo:hi].reshape((a.shape[0],) + R.PARAM_SHAPES[k]), dtype=torch.float32,
                               device="cuda").contiguous() for k, (lo, hi) in COLS.items()}


def _join(d, rows):
    return np.concatenate([to_np(d[k]).reshape(rows, -1) for k in COLS], axis=1)


@pytest.mark.parametrize("n,frac,steps", [(40_000, 0.1, 3), (1000, 0.0, 1), (777, 1.0, 2)])
def test_sparse_adam_matches_oracle(n, frac, steps):
    rng = np.random.default_rng(n)
    mask = scenes.random_active_mask(n, frac, n + 1) if 0 < frac < 1 else np.full(n, 1 if frac else 0, np.uint8)
    idx = np.where(mask)[0]
    r = R.Renderer(n, [(16, 16)])
    r.set_active(torch.as_tensor(mask, device="cuda"))
    p0 = rng.normal(size=(n, 75)).astype(np.float32)
    m0 = (rng.normal(size=(n, 75)) * 1e-3).astype(np.float32)
    v0 = (rng.random((n, 75)) * 1e-6).astype(np.float32)
    P, M, V = _split(p0, n), _split(m0, n), _split(v0, n)
    for d, val in ((P, 6.0), (M, 0.01), (V, 1e-4)):
        d["sigma"] = torch.tensor([val], dtype=torch.float32, device="cuda")
    lr = [1.6e-4, 1e-3, 5e-3, 1e-2, 2.5e-3, 1.25e-4, 5e-3, 0.1]
    # the oracle takes the hyper-parameters the library receives: FP32 values (0.999 is not one)
    f32 = lambda x: float(np.float32(x))  # noqa: E731
    lr32 = [f32(x) for x in lr]
    b1, b2, ep = f32(0.9), f32(0.999), f32(1e-15)
    ref = (p0.astype(np.float64), m0.astype(np.float64), v0.astype(np.float64))
    sig = (6.0, 0.01, 1e-4)
    mabs = np.abs(m0).astype(np.float64)  # the moment recursion over absolute values: the scale of m's rounding
    for t in range(1, steps + 1):
        g = (rng.normal(size=(len(idx), 75)) * 10.0 ** rng.integers(-4, 1, size=(len(idx), 1))).astype(np.float32)
        G = _split(g, len(idx)) if len(idx) else {k: torch.zeros((0,) + R.PARAM_SHAPES[k], device="cuda")
                                                   for k in COLS}
        G["sigma"] = torch.tensor([0.37 * t], dtype=torch.float32, device="cuda")
        r.adam_step(G, P, M, V, lr, t, eps=1e-15)
        ref = oad.sparse_adam(*ref, g.astype(np.float64), idx, lr32, t, b1, b2, ep)
        mabs[idx] = b1 * mabs[idx] + (1 - b1) * np.abs(g.astype(np.float64))
        ps, ms, vs = oad.adam_rows(np.array([sig[0]]), np.array([sig[1]]), np.array([sig[2]]),
                                   np.array([np.float32(0.37 * t)], dtype=np.float64), lr32[7], t, b1, b2, ep)
        sig = (ps[0], ms[0], vs[0])
    torch.cuda.synchronize()
    r.status()
    gp, gm, gv = _join(P, n), _join(M, n), _join(V, n)
    lr_col = np.asarray(lr32)[oad.COLUMN_RATE][None, :]
    # FP32 step: a few roundings of each Adam operation, relative to the step size; the stored p rounds too
    assert np.all(np.abs(gp - ref[0]) <= 1e-5 * lr_col * steps + 2e-7 * np.abs(ref[0]))
    # m: the update can cancel (b1 m and (1 - b1) g of opposite signs), so its error scales with mabs
    assert np.all(np.abs(gm - ref[1]) <= 1e-6 * mabs * steps)
    assert np.all(np.abs(gv - ref[2]) <= 1e-6 * np.abs(ref[2]) + 1e-18)
    rest = np.setdiff1d(np.arange(n), idx)
    assert np.array_equal(gp[rest], p0[rest]) and np.array_equal(gm[rest], m0[rest]) and \
        np.array_equal(gv[rest], v0[rest])
    assert abs(P["sigma"].item() - sig[0]) <= 1e-5 * lr[7] * steps + 1e-6 * abs(sig[0])
