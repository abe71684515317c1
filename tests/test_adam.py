"""Sparse Adam oracle (Sec. 5.1 Adam; Sec. 4.1 active set only) against
torch.optim.Adam in float64 and the first-step closed form (no GPU)."""
import numpy as np
import torch

from oracle import adam as oad


def test_matches_torch_adam_float64_over_steps():
    rng = np.random.default_rng(0)
    n = 6
    p0 = rng.normal(size=(n, 75))
    lr = [1.6e-4, 1e-3, 5e-3, 1e-2, 2.5e-3, 1.25e-4, 5e-3, 0.1]
    lr_col = np.asarray(lr)[oad.COLUMN_RATE]
    # torch: one parameter tensor per column rate class so each gets its own lr
    tp = torch.tensor(p0, dtype=torch.float64)
    leaves = [tp[:, oad.COLUMN_RATE == k].clone().requires_grad_(True) for k in range(7)]
    opt = torch.optim.Adam([{"params": [leaves[k]], "lr": lr[k]} for k in range(7)], betas=(0.9, 0.999), eps=1e-8)
    P, M, V = p0.copy(), np.zeros_like(p0), np.zeros_like(p0)
    for t in range(1, 6):
        g = rng.normal(size=(n, 75)) * 10.0 ** rng.integers(-3, 2, size=(n, 1))
        for k in range(7):
            leaves[k].grad = torch.tensor(g[:, oad.COLUMN_RATE == k])
        opt.step()
        P, M, V = oad.sparse_adam(P, M, V, g, np.arange(n), lr, t, 0.9, 0.999, 1e-8)
    got = np.zeros_like(p0)
    for k in range(7):
        got[:, oad.COLUMN_RATE == k] = leaves[k].detach().numpy()
    assert np.allclose(P, got, rtol=0, atol=1e-13)
    assert lr_col.shape == (75,)


def test_first_step_moves_each_element_by_its_rate():
    # t = 1: m = (1 - b1) g and v = (1 - b2) g^2 give |step| = lr |g| / (|g| + eps sqrt(1 - b2)) ~ lr
    rng = np.random.default_rng(1)
    p0 = rng.normal(size=(3, 75))
    g = rng.normal(size=(3, 75))
    lr = [1e-3, 2e-3, 3e-3, 4e-3, 5e-3, 6e-3, 7e-3, 0.1]
    P, _, _ = oad.sparse_adam(p0, np.zeros_like(p0), np.zeros_like(p0), g, np.arange(3), lr, 1)
    want = np.asarray(lr)[oad.COLUMN_RATE][None, :] * np.sign(g)
    assert np.allclose(p0 - P, want, rtol=1e-9, atol=0)
    # the colour SH degree-0 columns (11, 12, 13) take rate class 4, the rest of the colour SH class 5
    assert list(oad.COLUMN_RATE[11:15]) == [4, 4, 4, 5] and oad.COLUMN_RATE[58] == 5 and oad.COLUMN_RATE[59] == 6


def test_inactive_rows_untouched():
    rng = np.random.default_rng(2)
    p0, m0, v0 = rng.normal(size=(10, 75)), rng.random((10, 75)), rng.random((10, 75))
    idx = np.array([1, 4, 7])
    P, M, V = oad.sparse_adam(p0, m0, v0, rng.normal(size=(3, 75)), idx, [1e-3] * 8, 3)
    rest = np.setdiff1d(np.arange(10), idx)
    assert np.array_equal(P[rest], p0[rest]) and np.array_equal(M[rest], m0[rest]) and np.array_equal(V[rest], v0[rest])
    assert not np.any(P[idx] == p0[idx])
