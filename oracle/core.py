"""ctypes wrapper of ``sparseoit_oracle.c`` (FP64 CPU oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).  The C file is
compiled with gcc on first use, or by ``build()``.  All inputs are converted
to contiguous float64 numpy arrays; nothing here touches a GPU.

Parameter layout (per splat, the same as the library's inputs):
  means [N,3], quats [N,4] (w, x, y, z; need not be unit), log_scales [N,3],
  opacity_logits [N], sh_color [N,16,3], sh_weight [N,16];
  scalar sigma (Eq. 1) and background c0 [3] (Eq. 7).
Camera: dict with R [3,3] (world -> camera, x right, y down, z forward),
  t [3], fx, fy, cx, cy, width, height.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sparseoit_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NPARAM = 75  # mean 3, quat 4, log-scale 3, opacity logit 1, colour SH 48, weight SH 16

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, OpenMP)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.oracle_sh_basis.argtypes = [_dp, _dp, _dp]
            lib.oracle_sh_basis.restype = None
            params = [ctypes.c_int64, _dp, _dp, _dp, _dp, _dp, _dp, ctypes.c_double]
            lib.oracle_project.argtypes = params + [_dp, ctypes.c_int, ctypes.c_int, _dp]
            lib.oracle_project.restype = ctypes.c_int
            lib.oracle_render_sums.argtypes = params + [
                _dp, ctypes.c_int, ctypes.c_int, _u8p, ctypes.c_int, _ip, ctypes.c_double, _dp, _ip, _i64p, _dp]
            lib.oracle_render_sums.restype = ctypes.c_int
            lib.oracle_compose.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp]
            lib.oracle_compose.restype = ctypes.c_int
            lib.oracle_backward.argtypes = params + [
                _dp, _dp, ctypes.c_int, ctypes.c_int, _u8p, _dp, _dp, _ip, ctypes.c_double, _dp, _dp, _u8p, _dp]
            lib.oracle_backward.restype = ctypes.c_int
            lib.oracle_num_threads.argtypes = []
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a, t=_dp):
    return None if a is None else a.ctypes.data_as(t)


def _cam16(cam):
    c = np.zeros(16, dtype=np.float64)
    c[:9] = np.asarray(cam["R"], dtype=np.float64).reshape(9)
    c[9:12] = np.asarray(cam["t"], dtype=np.float64).reshape(3)
    c[12:16] = [cam["fx"], cam["fy"], cam["cx"], cam["cy"]]
    return c


def _splat_args(scene):
    n = int(np.asarray(scene["means"]).shape[0])
    arrs = [_f64(scene["means"]).reshape(n, 3), _f64(scene["quats"]).reshape(n, 4),
            _f64(scene["log_scales"]).reshape(n, 3), _f64(scene["opacity_logits"]).reshape(n),
            _f64(scene["sh_color"]).reshape(n, 16, 3), _f64(scene["sh_weight"]).reshape(n, 16)]
    return n, arrs


def _mask(mask, n):
    if mask is None:
        return None
    m = np.ascontiguousarray(np.asarray(mask).astype(np.uint8).reshape(n))
    return m


def _window(window):
    if window is None:
        return None
    return np.ascontiguousarray(np.asarray(window, dtype=np.int32).reshape(4))


def sh_basis(n):
    """Real SH basis Y[16] at unit direction n and its polynomial gradient dY[16,3]."""
    lib = _load()
    nn = _f64(n).reshape(3)
    Y = np.zeros(16)
    dY = np.zeros((16, 3))
    lib.oracle_sh_basis(_ptr(nn), _ptr(Y), _ptr(dY))
    return Y, dY


def project(scene, cam):
    """Per-splat projection, float64 [N, 24]; column layout in sparseoit_oracle.c."""
    lib = _load()
    n, a = _splat_args(scene)
    out = np.zeros((n, 24))
    c = _cam16(cam)
    lib.oracle_project(n, *[_ptr(x) for x in a], float(scene["sigma"]), _ptr(c),
                       int(cam["width"]), int(cam["height"]), _ptr(out))
    return out


def render_sums(scene, cam, subset=None, brute=False, window=None, amb_band=0.0, want_amb=False,
                amb_sums=None):
    """Per-pixel sums (P_r, P_g, P_b, Q, log T) of the selected splats, float64 [5, H, W].

    Returns (sums, amb_pixel or None, stats) where stats = (contributing pairs, clamped pairs).
    amb_sums (optional float64 [3, H, W]) receives, over the pairs within amb_band of the 1/255
    cut, sum a/(1-a), sum a w and sum a w max_c c.
    """
    lib = _load()
    n, a = _splat_args(scene)
    W, H = int(cam["width"]), int(cam["height"])
    sums = np.zeros((5, H, W))
    amb = np.zeros((H, W), dtype=np.int32) if want_amb else None
    stats = np.zeros(2, dtype=np.int64)
    m = _mask(subset, n)
    win = _window(window)
    c = _cam16(cam)
    if amb_sums is not None:
        assert amb_sums.dtype == np.float64 and amb_sums.shape == (3, H, W) and amb_sums.flags.c_contiguous
    rc = lib.oracle_render_sums(n, *[_ptr(x) for x in a], float(scene["sigma"]), _ptr(c), W, H,
                                _ptr(m, _u8p), int(bool(brute)), _ptr(win, _ip), float(amb_band),
                                _ptr(sums), _ptr(amb, _ip), _ptr(stats, _i64p), _ptr(amb_sums))
    if rc != 0:
        raise MemoryError("oracle_render_sums failed")
    return sums, amb, (int(stats[0]), int(stats[1]))


def compose(sums, bg):
    """Eq. 7 from sums [5,H,W]: image [H,W,3] and aux [H,W,5] = (F_r, F_g, F_b, T, Q)."""
    lib = _load()
    s = _f64(sums)
    _, H, W = s.shape
    img = np.zeros((H, W, 3))
    aux = np.zeros((H, W, 5))
    b = _f64(bg).reshape(3)
    lib.oracle_compose(W, H, _ptr(s), _ptr(b), _ptr(img), _ptr(aux))
    return img, aux


def render(scene, cam, subset=None, frozen_sums=None, brute=False, window=None, amb_band=0.0,
           frozen_amb_sums=None):
    """Image of the selected splats plus optional extra sums (e.g. a frozen complement).

    Returns dict(image [H,W,3], sums [5,H,W] (total), amb [H,W] int32, flip [H,W], pairs, clamped).
    flip bounds, to first order, how far the pairs within amb_band of the 1/255 cut can move the
    pixel's colour (in any channel) if included or dropped:
        T max|F - c0| sum a/(1-a) + (1 - T)/Q (sum a w max c + max|F| sum a w),
    and (1 - T) (max c + max|F|) where those pairs hold at least half of Q.
    frozen_amb_sums adds the same sums of a frozen complement rendered separately.
    """
    W, H = int(cam["width"]), int(cam["height"])
    ab = np.zeros((3, H, W))
    sums, amb, (pairs, clamped) = render_sums(scene, cam, subset, brute, window, amb_band, True, ab)
    if frozen_sums is not None:
        sums = sums + _f64(frozen_sums)
    if frozen_amb_sums is not None:
        ab = ab + _f64(frozen_amb_sums)
    img, aux = compose(sums, scene["bg"])
    F, T, Q = aux[..., :3], aux[..., 3], aux[..., 4]
    bg = _f64(scene["bg"]).reshape(3)
    fmax = np.abs(F).max(axis=2)
    fc0 = np.abs(F - bg).max(axis=2)
    with np.errstate(divide="ignore", invalid="ignore"):
        flip = T * fc0 * ab[0] + np.where(Q > 0, (1 - T) / np.where(Q > 0, Q, 1) * (ab[2] + fmax * ab[1]), 0.0)
    heavy = ab[1] >= 0.5 * Q
    cmax = np.where(ab[1] > 0, ab[2] / np.where(ab[1] > 0, ab[1], 1), 0.0)
    flip = np.where(heavy & (ab[1] > 0), np.maximum(flip, (1 - T) * (cmax + fmax)), flip)
    return dict(image=img, sums=sums, aux=aux, amb=amb, flip=flip, pairs=pairs, clamped=clamped)


def backward_full(scene, cam, sums_total, dL_dC, active=None, window=None, amb_band=0.0, want_flip=False):
    """Analytic gradient of L = sum dL_dC . C (Eq. 10 chained to all parameters).

    Returns dict(grads [N,75] (unselected rows NaN), dsigma, dsigma_scale (sum of |per-splat terms|),
    amb [N] uint8 (bit 0: a pair near the 1/255 cut or the 0.99 clamp; bit 1: a max(0,.) kink or the
    near plane within amb_band), flip [N,75] (sum over the bit-0 pairs of |that pair's gradient|,
    with want_flip) and dsigma_flip)."""
    lib = _load()
    n, a = _splat_args(scene)
    W, H = int(cam["width"]), int(cam["height"])
    s = _f64(sums_total).reshape(5, H, W)
    g = _f64(dL_dC).reshape(H, W, 3)
    grads = np.full((n, NPARAM), np.nan)
    flip = np.zeros((n, NPARAM)) if want_flip else None
    dsig = np.zeros(3)
    amb = np.zeros(n, dtype=np.uint8)
    m = _mask(active, n)
    win = _window(window)
    b = _f64(scene["bg"]).reshape(3)
    c = _cam16(cam)
    lib.oracle_backward(n, *[_ptr(x) for x in a], float(scene["sigma"]), _ptr(b), _ptr(c), W, H,
                        _ptr(m, _u8p), _ptr(s), _ptr(g), _ptr(win, _ip), float(amb_band),
                        _ptr(grads), _ptr(dsig), _ptr(amb, _u8p), _ptr(flip))
    return dict(grads=grads, dsigma=float(dsig[0]), dsigma_scale=float(dsig[1]), dsigma_flip=float(dsig[2]),
                amb=amb, flip=flip)


def backward(scene, cam, sums_total, dL_dC, active=None, window=None, amb_band=0.0, with_scale=False):
    """Analytic gradient of L = sum dL_dC . C (Eq. 10 chained to all parameters).

    Returns (grads [N,75] with unselected rows NaN, dL/dsigma, amb_splat [N] uint8 (nonzero: some
    ambiguity within amb_band, see backward_full)), and with with_scale=True a fourth value: the
    sum of |per-splat dL/dsigma terms|.
    """
    r = backward_full(scene, cam, sums_total, dL_dC, active, window, amb_band)
    if with_scale:
        return r["grads"], r["dsigma"], r["amb"], r["dsigma_scale"]
    return r["grads"], r["dsigma"], r["amb"]
