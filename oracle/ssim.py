"""FP64 oracle of the 3DGS photometric loss L = (1 - lambda) L1 + lambda (1 - SSIM).

TEST INFRASTRUCTURE ONLY (see the package docstring).  The paper keeps the
loss and its weight of the original 3DGS (Sec. 5.1, "Implementation
Details"): SSIM of Wang et al. (2004) per colour channel with an 11 x 11
Gaussian window of sigma 1.5, zero padding outside the image ("same"
output), C1 = 0.01^2, C2 = 0.03^2, averaged over all pixels and channels;
lambda = 0.2.  Written from the definition:
  mu_x = G * x, s_xx = G * x^2 - mu_x^2, s_xy = G * (x y) - mu_x mu_y,
  S = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_xx + s_yy + C2)).
The gradient of sum(S) with respect to x: with a = dS/dmu_x, b = dS/dE[x^2],
c = dS/dE[xy] taken per output pixel (E[.] = G * .),
  d sum(S)/dx = G^T * a + 2 x (G^T * b) + y (G^T * c),
and G^T * is the same zero-padded filtering since the window is symmetric.
"""
import numpy as np

WINDOW = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2
LAMBDA = 0.2


def window_1d(size=WINDOW, sigma=SIGMA) -> np.ndarray:
    x = np.arange(size, dtype=np.float64) - (size // 2)
    g = np.exp(-x * x / (2.0 * sigma * sigma))
    return g / g.sum()


def filt(img: np.ndarray, w1=None) -> np.ndarray:
    """Zero-padded 'same' 2D filtering of [H, W] with the separable Gaussian window (rows, then columns)."""
    w1 = window_1d() if w1 is None else w1
    r = len(w1) // 2
    H, W = img.shape
    p = np.zeros((H + 2 * r, W + 2 * r))
    p[r:r + H, r:r + W] = img
    tmp = np.zeros((H + 2 * r, W))
    for k in range(len(w1)):
        tmp += w1[k] * p[:, k:k + W]
    out = np.zeros((H, W))
    for k in range(len(w1)):
        out += w1[k] * tmp[k:k + H, :]
    return out


def ssim_maps(x2: np.ndarray, y2: np.ndarray):
    """One channel: (S map, a, b, c) as in the module docstring."""
    mx, my = filt(x2), filt(y2)
    exx, eyy, exy = filt(x2 * x2), filt(y2 * y2), filt(x2 * y2)
    sxx, syy, sxy = exx - mx * mx, eyy - my * my, exy - mx * my
    A = 2 * mx * my + C1
    B = 2 * sxy + C2
    Cc = mx * mx + my * my + C1
    D = sxx + syy + C2
    S = A * B / (Cc * D)
    a = S * (2 * my / A - 2 * my / B - 2 * mx / Cc + 2 * mx / D)
    b = -S / D
    c = 2 * S / B
    return S, a, b, c


def ssim(img: np.ndarray, target: np.ndarray) -> float:
    """Mean SSIM over [H, W, 3]."""
    return float(np.mean([ssim_maps(img[..., k].astype(np.float64), target[..., k].astype(np.float64))[0]
                          for k in range(img.shape[2])]))


def loss_l1_dssim(img: np.ndarray, target: np.ndarray, lam=LAMBDA) -> float:
    x, y = np.asarray(img, np.float64), np.asarray(target, np.float64)
    return float((1 - lam) * np.mean(np.abs(x - y)) + lam * (1.0 - ssim(x, y)))


def grad_l1_dssim(img: np.ndarray, target: np.ndarray, lam=LAMBDA) -> np.ndarray:
    """dL/dC for [H, W, 3] (sign(0) = 0 for the L1 part)."""
    x, y = np.asarray(img, np.float64), np.asarray(target, np.float64)
    n = x.size
    g = (1 - lam) * np.sign(x - y) / n
    for k in range(x.shape[2]):
        _, a, b, c = ssim_maps(x[..., k], y[..., k])
        dS = filt(a) + 2 * x[..., k] * filt(b) + y[..., k] * filt(c)
        g[..., k] -= lam * dS / n
    return g
