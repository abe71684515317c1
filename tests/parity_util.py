"""Comparison helpers for the GPU-vs-oracle parity tests.

Tolerances (stated for the FP32 CUDA path against the FP64 oracle):
  * image: max |C_gpu - C_ref| / max |C_ref| <= 1e-5 over the pixels of a
    view, excluding pixels where some splat's unclamped alpha lies within a
    relative AMB_BAND of the 1/255 cut (there FP32 and FP64 may disagree on
    whether the splat contributes at all; AMB_BAND = 1e-4 covers the FP32
    error of the exponent at the cutoff edge of a small splat, ~6e-5 px of
    centre rounding over a 2 px sigma; such pixels must stay below
    AMB_PIX_MAX of the view);
  * gradients: per parameter group, max |g_gpu - g_ref| / max |g_ref|
    <= 1e-4, excluding splats with a pair within AMB_BAND of the 1/255 cut or
    the 0.99 clamp, or a kink of max(0, .) (colour, weight, 1 - z/sigma)
    within AMB_BAND.
"""
import numpy as np
import torch

IMG_TOL = 1e-5
GRAD_TOL = 1e-4
AMB_BAND = 1e-4
AMB_PIX_MAX = 1e-2

GROUPS = dict(means=(0, 3), quats=(3, 7), log_scales=(7, 10), opacity_logits=(10, 11), sh_color=(11, 59),
              sh_weight=(59, 75))


def to_np(t):
    return t.detach().float().cpu().numpy().astype(np.float64)


def image_error(img_gpu, ref_img, amb=None):
    a = to_np(img_gpu) if isinstance(img_gpu, torch.Tensor) else img_gpu
    keep = np.ones(a.shape[:2], bool) if amb is None else (amb == 0)
    scale = max(np.abs(ref_img).max(), 1e-30)
    return float(np.abs(a - ref_img)[keep].max(initial=0.0) / scale), float(1.0 - keep.mean())


def grad_errors(gpu: dict, ref: np.ndarray, rows: np.ndarray, keep: np.ndarray):
    """gpu: dict of group -> array [len(rows), ...] in the order of `rows`;
    ref: oracle grads [N, 75]; keep: bool over rows."""
    out = {}
    for name, (lo, hi) in GROUPS.items():
        g = to_np(gpu[name]).reshape(len(rows), -1)[keep]
        r = ref[rows][keep, lo:hi]
        scale = max(np.abs(r).max(initial=0.0), 1e-30)
        out[name] = float(np.abs(g - r).max(initial=0.0) / scale)
    return out


def assert_grads_close(gpu, ref, rows, keep, tol=GRAD_TOL, dsig=None, dsig_ref=None, dsig_scale=None):
    """Per-group normwise check; dL/dsigma (a sum over splats whose terms
    cancel) is measured against the sum of the absolute terms."""
    errs = grad_errors(gpu, ref, rows, keep)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, f"gradient parity failed: {errs}"
    if dsig is not None:
        scale = dsig_scale if dsig_scale is not None else abs(dsig_ref)
        rel = abs(dsig - dsig_ref) / max(scale, 1e-30)
        errs["sigma"] = rel
        assert rel <= tol, f"dsigma {dsig} vs {dsig_ref} (rel {rel:.3g} of {scale:.3g})"
    return errs
