"""The D-SSIM loss oracle (3DGS loss, kept by the paper, Sec. 5.1) against
library routines, identities and finite differences (no GPU)."""
import numpy as np
import pytest
from scipy import ndimage, signal

from oracle import ssim as osm


def test_window_is_scipy_gaussian():
    w = signal.windows.gaussian(11, 1.5)
    assert np.allclose(osm.window_1d(), w / w.sum(), atol=1e-15)


def test_filter_is_zero_padded_correlation():
    rng = np.random.default_rng(0)
    img = rng.random((23, 17))
    w = osm.window_1d()
    ref = ndimage.correlate(img, np.outer(w, w), mode="constant", cval=0.0)
    assert np.allclose(osm.filt(img), ref, atol=1e-14)


def test_identities():
    rng = np.random.default_rng(1)
    x, y = rng.random((20, 24, 3)), rng.random((20, 24, 3))
    assert abs(osm.ssim(x, x) - 1.0) < 1e-12
    assert abs(osm.ssim(x, y) - osm.ssim(y, x)) < 1e-12
    assert osm.ssim(x, y) < 0.5
    assert abs(osm.loss_l1_dssim(x, x)) < 1e-12
    # a perfect match is a stationary point of the SSIM term
    g = osm.grad_l1_dssim(x, x)
    assert np.abs(g).max() < 1e-12


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(2)
    x, y = rng.random((12, 14, 3)), rng.random((12, 14, 3))
    g = osm.grad_l1_dssim(x, y)
    for (i, j, k) in [(0, 0, 0), (5, 7, 1), (11, 13, 2), (6, 0, 0), (3, 9, 2), (11, 2, 1)]:
        h = 1e-6
        xp, xm = x.copy(), x.copy()
        xp[i, j, k] += h
        xm[i, j, k] -= h
        fd = (osm.loss_l1_dssim(xp, y) - osm.loss_l1_dssim(xm, y)) / (2 * h)
        assert abs(fd - g[i, j, k]) <= 1e-7 * max(1.0, abs(fd)), (i, j, k, fd, g[i, j, k])


def test_pure_ssim_term_gradient_and_lambda():
    rng = np.random.default_rng(3)
    x, y = rng.random((9, 10, 3)), rng.random((9, 10, 3))
    # lambda = 0 is the plain L1 mean; lambda = 1 the pure D-SSIM
    assert np.isclose(osm.loss_l1_dssim(x, y, 0.0), np.mean(np.abs(x - y)))
    assert np.isclose(osm.loss_l1_dssim(x, y, 1.0), 1.0 - osm.ssim(x, y))
    g1 = osm.grad_l1_dssim(x, y, 1.0)
    h = 1e-6
    xp, xm = x.copy(), x.copy()
    xp[4, 5, 1] += h
    xm[4, 5, 1] -= h
    fd = ((1 - osm.ssim(xp, y)) - (1 - osm.ssim(xm, y))) / (2 * h)
    assert abs(fd - g1[4, 5, 1]) < 1e-8


def test_closed_form_on_a_checkerboard_against_a_constant():
    # x = a + d (-1)^(i+j), y = b: at an interior pixel mu_x = a + d s c^2 (s = (-1)^(i+j),
    # c = sum_k w_k (-1)^(k-5)), E[x^2] = a^2 + 2 a d s c^2 + d^2, so s_xx = d^2 (1 - c^4);
    # mu_y = b, s_yy = 0, s_xy = 0: S = (2 mu_x b + C1) C2 / ((mu_x^2 + b^2 + C1)(s_xx + C2))
    a, d, b = 0.4, 0.1, 0.7
    n = 31
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    x = a + d * (-1.0) ** (i + j)
    y = np.full((n, n), b)
    S, _, _, _ = osm.ssim_maps(x, y)
    w = osm.window_1d()
    c = np.sum(w * (-1.0) ** (np.arange(11) - 5))
    for (p, q) in [(15, 15), (12, 17), (8, 9)]:
        s = (-1.0) ** (p + q)
        mx = a + d * s * c * c
        sxx = d * d * (1 - c ** 4)
        want = (2 * mx * b + osm.C1) * osm.C2 / ((mx * mx + b * b + osm.C1) * (sxx + osm.C2))
        assert abs(S[p, q] - want) < 1e-12, (p, q, S[p, q], want)
    # the constants are those of 3DGS (data range 1)
    assert osm.C1 == 0.01 ** 2 and osm.C2 == 0.03 ** 2 and osm.LAMBDA == 0.2
