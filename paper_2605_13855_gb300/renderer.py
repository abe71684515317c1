"""Python binding of libsparseoit: argument marshalling only.

Every step of the renderer runs in the library's CUDA kernels; this module
passes device pointers of PyTorch tensors and the current CUDA stream
through the C ABI (include/sparseoit.h).  PyTorch supplies device memory,
streams and autograd plumbing.  There is no CPU fallback: without the built
library or a CUDA device every call raises.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from . import _lib
from ._lib import SparseOITError

PARAM_NAMES = ("means", "quats", "log_scales", "opacity_logits", "sh_color", "sh_weight")
PARAM_SHAPES = {"means": (3,), "quats": (4,), "log_scales": (3,), "opacity_logits": (), "sh_color": (16, 3),
                "sh_weight": (16,)}


@dataclass
class SplatParams:
    """Splat parameters on the GPU (Sec. 3.1 / 3.2; Eq. 1 sigma, Eq. 7 c0)."""
    means: torch.Tensor           # [N, 3] float32
    quats: torch.Tensor           # [N, 4] float32 (w, x, y, z)
    log_scales: torch.Tensor      # [N, 3] float32
    opacity_logits: torch.Tensor  # [N]    float32
    sh_color: torch.Tensor        # [N, 16, 3] float32 or bfloat16
    sh_weight: torch.Tensor       # [N, 16]    float32 or bfloat16
    sigma: float = 6.0
    bg: Sequence[float] = field(default_factory=lambda: (0.0, 0.0, 0.0))
    active_rows: bool = False     # rows are the active splats in active order (Renderer.gather_active)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @staticmethod
    def from_numpy(scene: dict, device="cuda", sh_dtype=torch.float32) -> "SplatParams":
        def t(a, dt=torch.float32):
            return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).to(device=device, dtype=dt)
        return SplatParams(t(scene["means"]), t(scene["quats"]), t(scene["log_scales"]),
                           t(scene["opacity_logits"]), t(scene["sh_color"], sh_dtype), t(scene["sh_weight"], sh_dtype),
                           float(scene["sigma"]), tuple(float(x) for x in scene["bg"]))


def _check_param(name, t: torch.Tensor, n: int):
    want = (n,) + PARAM_SHAPES[name]
    if tuple(t.shape) != want:
        raise ValueError(f"{name}: shape {tuple(t.shape)} != {want}")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def splats_struct(p: SplatParams) -> _lib.Splats:
    n = p.n
    for name in PARAM_NAMES:
        _check_param(name, getattr(p, name), n)
    for name in ("means", "quats", "log_scales", "opacity_logits"):
        if getattr(p, name).dtype != torch.float32:
            raise ValueError(f"{name} must be float32")
    if p.sh_color.dtype != p.sh_weight.dtype or p.sh_color.dtype not in (torch.float32, torch.bfloat16):
        raise ValueError("sh_color / sh_weight must both be float32 or both bfloat16")
    s = _lib.Splats()
    s.means = p.means.data_ptr()
    s.quats = p.quats.data_ptr()
    s.log_scales = p.log_scales.data_ptr()
    s.opacity_logits = p.opacity_logits.data_ptr()
    s.sh_color = p.sh_color.data_ptr()
    s.sh_weight = p.sh_weight.data_ptr()
    s.sh_dtype = _lib.BF16 if p.sh_color.dtype == torch.bfloat16 else _lib.F32
    s.sigma = float(p.sigma)
    for k in range(3):
        s.bg[k] = float(p.bg[k])
    s.n = n
    s.rows = _lib.ROWS_ACTIVE if p.active_rows else _lib.ROWS_BY_SPLAT
    return s


def camera_struct(cam: dict) -> _lib.Camera:
    c = _lib.Camera()
    R = np.asarray(cam["R"], dtype=np.float32).reshape(9)
    t = np.asarray(cam["t"], dtype=np.float32).reshape(3)
    for k in range(9):
        c.R[k] = float(R[k])
    for k in range(3):
        c.t[k] = float(t[k])
    c.fx, c.fy, c.cx, c.cy = (float(cam["fx"]), float(cam["fy"]), float(cam["cx"]), float(cam["cy"]))
    c.width, c.height = int(cam["width"]), int(cam["height"])
    return c


class _DeviceArray:
    """Zero-copy view of library-owned device memory through __cuda_array_interface__."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = dict(shape=tuple(shape), typestr=typestr, data=(int(ptr), False),
                                             version=3, strides=None)


def _stream_ptr(stream: Optional[torch.cuda.Stream] = None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class Renderer:
    """A SparseOIT context: active set, per-view frozen sums, batched fwd / bwd."""

    def __init__(self, n_splats: int, view_sizes: Sequence[Sequence[int]], max_pairs: int = 0,
                 fwd_pixels_per_thread: int = 0, proj_lanes_per_splat: int = 0, bwd_walk: int = 0,
                 raster_tile_order: int = 0, bwd_parallel: int = 0, raster_persistent: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("sparseoit needs a CUDA device")
        self.lib = _lib.load()
        self.n = int(n_splats)
        self.view_sizes = [(int(w), int(h)) for (w, h) in view_sizes]
        nv = len(self.view_sizes)
        ws = (ctypes.c_int32 * nv)(*[w for w, _ in self.view_sizes])
        hs = (ctypes.c_int32 * nv)(*[h for _, h in self.view_sizes])
        cfg = _lib.Config()
        cfg.max_pairs = int(max_pairs)
        cfg.fwd_pixels_per_thread = int(fwd_pixels_per_thread)
        cfg.proj_lanes_per_splat = int(proj_lanes_per_splat)
        cfg.bwd_walk = int(bwd_walk)
        cfg.raster_tile_order = int(raster_tile_order)
        cfg.bwd_parallel = int(bwd_parallel)
        cfg.raster_persistent = int(raster_persistent)
        self._ctx = ctypes.c_void_p()
        rc = self.lib.sparseoit_create(ctypes.byref(self._ctx), self.n, nv, ws, hs, ctypes.byref(cfg))
        if rc != _lib.OK:
            raise SparseOITError(rc, self.lib.sparseoit_last_error(None).decode())
        self._n_active = 0
        self._pending_mask = None  # the mask of an asynchronous set_active, kept alive until its count is read
        self.forward_id = 0
        self._last_views: List[int] = []
        self._keep = None

    # ------------------------------------------------------------ basics
    def _check(self, rc):
        if rc != _lib.OK:
            raise SparseOITError(rc, self.lib.sparseoit_last_error(self._ctx).decode())

    def close(self):
        if getattr(self, "_ctx", None) is not None and self._ctx.value:
            self.lib.sparseoit_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------- active set
    def set_active(self, mask: torch.Tensor, stream=None, asynchronous: bool = False):
        """Sec. 4.1: set A from a [N] bool / uint8 CUDA mask.  By default the call synchronises the
        stream; asynchronous=True enqueues the compaction and returns, and |A| is read (waiting for
        that compaction only) when n_active or a later call first needs it."""
        if mask.dtype == torch.bool:
            mask = mask.to(torch.uint8)
        if mask.dtype != torch.uint8 or not mask.is_cuda or mask.numel() != self.n:
            raise ValueError("mask must be a CUDA uint8/bool tensor of n_splats entries")
        mask = mask.contiguous()
        fn = self.lib.sparseoit_set_active_async if asynchronous else self.lib.sparseoit_set_active
        self._check(fn(self._ctx, ctypes.c_void_p(mask.data_ptr()), self.n, ctypes.c_void_p(_stream_ptr(stream))))
        if asynchronous:
            self._pending_mask = mask
            self._n_active = None
        else:
            self._pending_mask = None
            self._read_n_active()

    def _read_n_active(self):
        p, na = ctypes.c_void_p(), ctypes.c_int64()
        self._check(self.lib.sparseoit_get_active(self._ctx, ctypes.byref(p), ctypes.byref(na)))
        self._n_active = int(na.value)
        self._pending_mask = None

    @property
    def n_active(self) -> int:
        """|A| of the current active set (after an asynchronous set_active: waits for its count)."""
        if self._n_active is None:
            self._read_n_active()
        return self._n_active

    def active_indices(self) -> torch.Tensor:
        """Ascending int32 indices of A (a copy)."""
        p, na = ctypes.c_void_p(), ctypes.c_int64()
        self._check(self.lib.sparseoit_get_active(self._ctx, ctypes.byref(p), ctypes.byref(na)))
        if na.value == 0:
            return torch.zeros(0, dtype=torch.int32, device="cuda")
        return torch.as_tensor(_DeviceArray(p.value, (na.value,), "<i4"), device="cuda").clone()

    def frozen_sums(self, view: int) -> torch.Tensor:
        """[5, H, W] frozen sums (P_r, P_g, P_b, Q, log T) of a view (a copy)."""
        p = ctypes.c_void_p()
        self._check(self.lib.sparseoit_get_frozen(self._ctx, int(view), ctypes.byref(p)))
        W, H = self.view_sizes[view]
        return torch.as_tensor(_DeviceArray(p.value, (5, H, W), "<f4"), device="cuda").clone()

    def set_frozen(self, view: int, planes: torch.Tensor, stream=None):
        """Restore a view's frozen sums ([5, H, W] float32, device or host, contiguous), e.g. saved by
        frozen_sums() under the same active set: checkpoint and resume without a recompute."""
        W, H = self.view_sizes[view]
        if planes.dtype != torch.float32 or tuple(planes.shape) != (5, H, W) or not planes.is_contiguous():
            raise ValueError(f"frozen planes must be contiguous float32 [5, {H}, {W}]")
        self._check(self.lib.sparseoit_set_frozen(self._ctx, int(view), ctypes.c_void_p(planes.data_ptr()),
                                                  ctypes.c_void_p(_stream_ptr(stream))))

    def commit_frozen(self, splats: SplatParams, cam: dict, view: int, mode: str = "incremental", stream=None):
        """Sec. 4.1 / Alg. 2 BAU: bring the view's frozen sums up to date."""
        m = _lib.COMMIT_INCREMENTAL if mode == "incremental" else _lib.COMMIT_RECOMPUTE
        s = splats_struct(splats)
        c = camera_struct(cam)
        self._check(self.lib.sparseoit_commit_frozen(self._ctx, ctypes.byref(s), ctypes.byref(c), int(view), m,
                                                     ctypes.c_void_p(_stream_ptr(stream))))

    # ------------------------------------------------------ forward / bwd
    def forward(self, splats: SplatParams, cams: Sequence[dict], views: Sequence[int],
                targets: Optional[Sequence[torch.Tensor]] = None, stream=None, images=None, loss=None):
        """Render the active set of the given views (Eq. 7 with the frozen sums).

        Returns (images list of [H, W, 3], loss tensor [1] or None)."""
        nv = len(views)
        if nv != len(cams) or nv < 1 or nv > _lib.MAX_BATCH_VIEWS:
            raise ValueError("need 1..32 views, one camera each")
        s = splats_struct(splats)
        camarr = (_lib.Camera * nv)(*[camera_struct(c) for c in cams])
        varr = (ctypes.c_int32 * nv)(*[int(v) for v in views])
        if images is None:
            images = [torch.empty((self.view_sizes[v][1], self.view_sizes[v][0], 3), dtype=torch.float32,
                                  device="cuda") for v in views]
        iptr = (ctypes.c_void_p * nv)(*[im.data_ptr() for im in images])
        tptr = None
        if targets is not None:
            for tg, v in zip(targets, views):
                W, H = self.view_sizes[v]
                if tuple(tg.shape) != (H, W, 3) or tg.dtype != torch.float32 or not tg.is_cuda \
                        or not tg.is_contiguous():
                    raise ValueError("targets must be contiguous float32 CUDA [H, W, 3]")
            tptr = (ctypes.c_void_p * nv)(*[tg.data_ptr() for tg in targets])
            if loss is None:
                loss = torch.empty(1, dtype=torch.float32, device="cuda")
        self._check(self.lib.sparseoit_forward(self._ctx, ctypes.byref(s), camarr, varr, nv, iptr, tptr,
                                               ctypes.c_void_p(loss.data_ptr() if loss is not None else 0),
                                               ctypes.c_void_p(_stream_ptr(stream))))
        self.forward_id += 1
        self._last_views = list(views)
        self._last_bg = tuple(float(x) for x in splats.bg)
        self._keep = (images, targets, loss)
        return images, loss

    def loss_l1_dssim(self, targets: Sequence[torch.Tensor], lam: float = 0.2, stream=None,
                      loss: Optional[torch.Tensor] = None, grad_images: Optional[Sequence[torch.Tensor]] = None):
        """(1 - lam) L1 + lam (1 - SSIM) of the last forward's images (run without targets) against
        `targets` (sparseoit_loss_l1_dssim); prepares the backward.  Returns the loss tensor [1]."""
        views = self._last_views
        if len(targets) != len(views):
            raise ValueError("one target per view of the last forward")
        for tg, v in zip(targets, views):
            W, H = self.view_sizes[v]
            if tuple(tg.shape) != (H, W, 3) or tg.dtype != torch.float32 or not tg.is_cuda or not tg.is_contiguous():
                raise ValueError("targets must be contiguous float32 CUDA [H, W, 3]")
        nv = len(views)
        tptr = (ctypes.c_void_p * nv)(*[tg.data_ptr() for tg in targets])
        gptr = None
        if grad_images is not None:
            gptr = (ctypes.c_void_p * nv)(*[g.data_ptr() for g in grad_images])
        if loss is None:
            loss = torch.empty(1, dtype=torch.float32, device="cuda")
        bg = (ctypes.c_float * 3)(*self._last_bg)
        self._check(self.lib.sparseoit_loss_l1_dssim(self._ctx, tptr, float(lam), ctypes.c_void_p(loss.data_ptr()),
                                                     gptr, bg, ctypes.c_void_p(_stream_ptr(stream))))
        self._keep_loss = (targets, grad_images, loss)
        return loss

    def backward(self, splats: SplatParams, grad_images: Optional[Sequence[torch.Tensor]] = None,
                 rows_by_splat: bool = False, stream=None, out: Optional[Dict[str, torch.Tensor]] = None,
                 accumulate: bool = False):
        """Gradients of the last forward's loss for the active splats (App. B).

        rows_by_splat=False: compact [n_active, ...] rows in active-index order;
        True: full [N, ...] arrays, inactive rows zero.  accumulate=True adds to `out`."""
        s = splats_struct(splats)
        rows = self.n if rows_by_splat else self.n_active
        if out is None:
            alloc = torch.zeros if rows_by_splat else torch.empty
            out = {name: alloc((rows,) + PARAM_SHAPES[name], dtype=torch.float32, device="cuda")
                   for name in PARAM_NAMES}
            out["sigma"] = torch.empty(1, dtype=torch.float32, device="cuda")
        g = _lib.Grads()
        for name in PARAM_NAMES + ("sigma",):
            setattr(g, name, out[name].data_ptr())
        g.rows_by_splat = 1 if rows_by_splat else 0
        g.accumulate = 1 if accumulate else 0
        gptr = None
        if grad_images is not None:
            gi = [x.contiguous().float() for x in grad_images]
            gptr = (ctypes.c_void_p * len(gi))(*[x.data_ptr() for x in gi])
            self._keep_grad = gi
        self._check(self.lib.sparseoit_backward(self._ctx, ctypes.byref(s), gptr, ctypes.byref(g),
                                                ctypes.c_void_p(_stream_ptr(stream))))
        return out

    def autotune(self, splats: SplatParams, cams: Sequence[dict], views: Sequence[int],
                 targets: Optional[Sequence[torch.Tensor]] = None, reps: int = 3, stream=None):
        """Pick the rasters' launch options for this batch (sparseoit_autotune): the forward strip and
        whether the forward runs as persistent blocks; with targets also the backward's splat order
        and persistence.

        Returns {"fwd_pixels_per_thread", "ms": {strip: mean forward ms}, "fwd_persistent",
        "fwd_persistent_ms", "bwd_walk", "bwd_persistent", "bwd_ms": {option: mean backward-raster ms}}."""
        nv = len(views)
        s = splats_struct(splats)
        camarr = (_lib.Camera * nv)(*[camera_struct(c) for c in cams])
        varr = (ctypes.c_int32 * nv)(*[int(v) for v in views])
        images = [torch.empty((self.view_sizes[v][1], self.view_sizes[v][0], 3), dtype=torch.float32, device="cuda")
                  for v in views]
        iptr = (ctypes.c_void_p * nv)(*[im.data_ptr() for im in images])
        tptr, loss = None, None
        if targets is not None:
            tptr = (ctypes.c_void_p * nv)(*[tg.data_ptr() for tg in targets])
            loss = torch.empty(1, dtype=torch.float32, device="cuda")
        t = _lib.Tuning()
        self._check(self.lib.sparseoit_autotune(self._ctx, ctypes.byref(s), camarr, varr, nv, iptr, tptr,
                                                ctypes.c_void_p(loss.data_ptr() if loss is not None else 0),
                                                int(reps), ctypes.byref(t), ctypes.c_void_p(_stream_ptr(stream))))
        self.forward_id += 1
        names = ("sorted", "arena", "sorted_persistent", "arena_persistent")
        return {"fwd_pixels_per_thread": int(t.fwd_pixels_per_thread),
                "ms": {int(t.candidates[k]): float(t.ms[k]) for k in range(t.n_candidates)},
                "fwd_persistent": int(t.fwd_persistent), "fwd_persistent_ms": float(t.fwd_persistent_ms),
                "bwd_walk": int(t.bwd_walk), "bwd_persistent": int(t.bwd_persistent),
                "bwd_ms": {names[k]: float(t.bwd_ms[k]) for k in range(4)} if t.bwd_walk else {}}

    def update_active_set(self, splats: SplatParams, cams: Sequence[dict], targets: Sequence[torch.Tensor],
                          eps: Sequence[float], n_sub: int, first: int, stream=None,
                          scratch: Optional[Dict[str, torch.Tensor]] = None, mask: Optional[torch.Tensor] = None):
        """The periodic active-set update (Sec. 4.1, Eq. 8; sparseoit_update_active_set).

        cams / targets: every training view of the context, in order.  Returns
        (mask u8 [N] on the device, picked views list, summed full-row gradients dict)."""
        nv = len(cams)
        if nv != len(self.view_sizes) or len(targets) != nv:
            raise ValueError("need one camera and one target per view of the renderer")
        s = splats_struct(splats)
        camarr = (_lib.Camera * nv)(*[camera_struct(c) for c in cams])
        for tg, (W, H) in zip(targets, self.view_sizes):
            if tuple(tg.shape) != (H, W, 3) or tg.dtype != torch.float32 or not tg.is_cuda or not tg.is_contiguous():
                raise ValueError("targets must be contiguous float32 CUDA [H, W, 3]")
        tptr = (ctypes.c_void_p * nv)(*[tg.data_ptr() for tg in targets])
        if scratch is None:
            scratch = {name: torch.empty((self.n,) + PARAM_SHAPES[name], dtype=torch.float32, device="cuda")
                       for name in PARAM_NAMES}
            scratch["sigma"] = torch.empty(1, dtype=torch.float32, device="cuda")
        g = _lib.Grads()
        for name in PARAM_NAMES + ("sigma",):
            setattr(g, name, scratch[name].data_ptr())
        if mask is None:
            mask = torch.empty(self.n, dtype=torch.uint8, device="cuda")
        epsa = (ctypes.c_float * 6)(*[float(e) for e in eps])
        sel = (ctypes.c_int32 * max(1, int(n_sub)))()
        self._check(self.lib.sparseoit_update_active_set(self._ctx, ctypes.byref(s), camarr, nv, tptr, int(n_sub),
                                                         int(first), epsa, ctypes.byref(g),
                                                         ctypes.c_void_p(mask.data_ptr()), sel,
                                                         ctypes.c_void_p(_stream_ptr(stream))))
        # the call ends with set_active on the new mask
        idx, na = ctypes.c_void_p(), ctypes.c_int64()
        self._check(self.lib.sparseoit_get_active(self._ctx, ctypes.byref(idx), ctypes.byref(na)))
        self._n_active = int(na.value)
        self._pending_mask = None
        self.forward_id += 1
        return mask, [int(sel[k]) for k in range(int(n_sub))], scratch

    def adam_step(self, grads: Dict[str, torch.Tensor], params: Dict[str, torch.Tensor], m: Dict[str, torch.Tensor],
                  v: Dict[str, torch.Tensor], lr: Sequence[float], step: int, beta1: float = 0.9,
                  beta2: float = 0.999, eps: float = 1e-15, stream=None):
        """Sparse Adam over the active rows (sparseoit_adam_step), in place on params / m / v.

        grads: compact rows of the last backward (active order); params, m, v: full rows by splat,
        or active rows (|A| rows, the layout of gather_active) -- dicts of FP32 CUDA tensors with the
        parameter names, plus optional "sigma" [1] in all four.
        lr: 8 rates (means, quats, log_scales, opacity, SH colour degree 0, degrees 1-3, SH weight, sigma)."""
        nrow = params["means"].shape[0]
        active_rows = nrow == self.n_active and nrow != self.n

        def rows(d):
            return self._rows_struct(d, nrow)
        g = _lib.Grads()
        for name in PARAM_NAMES:
            setattr(g, name, grads[name].data_ptr())
        g.sigma = grads["sigma"].data_ptr() if "sigma" in grads else 0
        rp, rm, rv = rows(params), rows(m), rows(v)
        cfg = _lib.Adam()
        if len(lr) != 8:
            raise ValueError("need 8 learning rates")
        for k in range(8):
            cfg.lr[k] = float(lr[k])
        cfg.beta1, cfg.beta2, cfg.eps, cfg.step = float(beta1), float(beta2), float(eps), int(step)
        cfg.rows = _lib.ROWS_ACTIVE if active_rows else _lib.ROWS_BY_SPLAT
        self._check(self.lib.sparseoit_adam_step(self._ctx, ctypes.byref(g), ctypes.byref(rp), ctypes.byref(rm),
                                                 ctypes.byref(rv), ctypes.byref(cfg),
                                                 ctypes.c_void_p(_stream_ptr(stream))))

    @staticmethod
    def _rows_struct(d: Dict[str, torch.Tensor], n: int, sh_dtype=None) -> "_lib.Rows":
        r = _lib.Rows()
        for name in PARAM_NAMES:
            t = d[name]
            want = torch.float32 if name not in ("sh_color", "sh_weight") or sh_dtype is None else sh_dtype
            if t.dtype != want or not t.is_cuda or not t.is_contiguous() or t.shape[0] != n:
                raise ValueError(f"{name} must be contiguous {want} CUDA with {n} rows")
            setattr(r, name, t.data_ptr())
        r.sigma = d["sigma"].data_ptr() if "sigma" in d else 0
        return r

    def gather_active(self, full: SplatParams, stream=None) -> SplatParams:
        """The active rows of `full` (rows by splat) as a new SplatParams in active order
        (sparseoit_gather_active): the stage layout read by forward / backward / adam_step."""
        na = self.n_active
        shdt = full.sh_color.dtype
        act = {name: torch.empty((na,) + PARAM_SHAPES[name], dtype=getattr(full, name).dtype, device="cuda")
               for name in PARAM_NAMES}
        src = self._rows_struct({k: getattr(full, k) for k in PARAM_NAMES}, self.n, shdt)
        dst = self._rows_struct(act, na, shdt)
        self._check(self.lib.sparseoit_gather_active(self._ctx, ctypes.byref(src), ctypes.byref(dst),
                                                     _lib.BF16 if shdt == torch.bfloat16 else _lib.F32,
                                                     ctypes.c_void_p(_stream_ptr(stream))))
        return SplatParams(*[act[k] for k in PARAM_NAMES], full.sigma, full.bg, active_rows=True)

    def scatter_active(self, active: SplatParams, full: SplatParams, stream=None):
        """Write the active rows back into `full` (sparseoit_scatter_active)."""
        shdt = full.sh_color.dtype
        src = self._rows_struct({k: getattr(active, k) for k in PARAM_NAMES}, self.n_active, shdt)
        dst = self._rows_struct({k: getattr(full, k) for k in PARAM_NAMES}, self.n, shdt)
        self._check(self.lib.sparseoit_scatter_active(self._ctx, ctypes.byref(src), ctypes.byref(dst),
                                                      _lib.BF16 if shdt == torch.bfloat16 else _lib.F32,
                                                      ctypes.c_void_p(_stream_ptr(stream))))

    # ------------------------------------------------------------ misc
    def status(self, stream=None):
        self._check(self.lib.sparseoit_status(self._ctx, ctypes.c_void_p(_stream_ptr(stream))))

    def inject_scan_stall(self, partition: int):
        """Failure injection (tests): the next binning's tile-scan partition `partition` posts
        nothing, so the later partitions' bounded waits run out (sparseoit_inject_scan_stall)."""
        self._check(self.lib.sparseoit_inject_scan_stall(self._ctx, int(partition)))

    def set_counting(self, enable: bool):
        self._check(self.lib.sparseoit_set_counting(self._ctx, 1 if enable else 0))

    def last_counts(self, stream=None):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.sparseoit_last_counts(self._ctx, ctypes.c_void_p(_stream_ptr(stream)),
                                                   ctypes.byref(a), ctypes.byref(b)))
        return int(a.value), int(b.value)

    def set_profiling(self, enable: bool):
        self._check(self.lib.sparseoit_set_profiling(self._ctx, 1 if enable else 0))

    def get_profile(self) -> Dict[str, tuple]:
        """{kernel: (launches, total_ms)} since the previous call (synchronises)."""
        buf = (_lib.KernelTime * 32)()
        n = ctypes.c_int32()
        self._check(self.lib.sparseoit_get_profile(self._ctx, 32, buf, ctypes.byref(n)))
        return {buf[k].name.decode(): (int(buf[k].launches), float(buf[k].total_ms)) for k in range(n.value)}

    def reserve_pairs(self, max_pairs: int):
        self._check(self.lib.sparseoit_reserve_pairs(self._ctx, int(max_pairs)))


class SparseOITRender(torch.autograd.Function):
    """Autograd wrapper: images of the active set; gradients for all rows
    (inactive rows zero), computed by sparseoit_backward."""

    @staticmethod
    def forward(ctx, renderer: Renderer, cams, views, sigma: float, bg, means, quats, log_scales, opacity_logits,
                sh_color, sh_weight):
        sp = SplatParams(means.detach(), quats.detach(), log_scales.detach(), opacity_logits.detach(),
                         sh_color.detach(), sh_weight.detach(), float(sigma), tuple(bg))
        images, _ = renderer.forward(sp, cams, views)
        ctx.renderer = renderer
        ctx.splats = sp
        ctx.forward_id = renderer.forward_id
        ctx.shapes = [tuple(im.shape) for im in images]
        return tuple(images)

    @staticmethod
    def backward(ctx, *grad_images):
        r: Renderer = ctx.renderer
        if r.forward_id != ctx.forward_id:
            raise RuntimeError("SparseOITRender.backward: another forward ran on this renderer since")
        gi = [g if g is not None else torch.zeros(shp, dtype=torch.float32, device="cuda")
              for g, shp in zip(grad_images, ctx.shapes)]
        grads = r.backward(ctx.splats, gi, rows_by_splat=True)
        sh_dt = ctx.splats.sh_color.dtype
        return (None, None, None, None, None, grads["means"], grads["quats"], grads["log_scales"],
                grads["opacity_logits"], grads["sh_color"].to(sh_dt), grads["sh_weight"].to(sh_dt))


def fps_views(cams: Sequence[dict], n_sub: int, first: int) -> List[int]:
    """Farthest point sampling of training views by camera centre (sparseoit_fps_views; host only)."""
    lib = _lib.load()
    n = len(cams)
    camarr = (_lib.Camera * n)(*[camera_struct(c) for c in cams])
    out = (ctypes.c_int32 * max(1, int(n_sub)))()
    rc = lib.sparseoit_fps_views(camarr, n, int(n_sub), int(first), out)
    if rc != _lib.OK:
        raise SparseOITError(rc, "fps_views: need 1 <= n_sub <= len(cams) and 0 <= first < len(cams)")
    return [int(out[k]) for k in range(int(n_sub))]


def activeness(grads: Dict[str, torch.Tensor], eps: Sequence[float], stream=None, with_norms: bool = False):
    """Eq. 8 on full gradient rows (sparseoit_activeness): (mask u8 [N], norms [N, 6] or None)."""
    lib = _lib.load()
    n = grads["means"].shape[0]
    g = _lib.Grads()
    for name in PARAM_NAMES:
        t = grads[name]
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or t.shape[0] != n:
            raise ValueError(f"gradient {name} must be contiguous float32 CUDA with {n} rows")
        setattr(g, name, t.data_ptr())
    mask = torch.empty(n, dtype=torch.uint8, device="cuda")
    norms = torch.empty((n, 6), dtype=torch.float32, device="cuda") if with_norms else None
    epsa = (ctypes.c_float * 6)(*[float(e) for e in eps])
    rc = lib.sparseoit_activeness(ctypes.byref(g), n, epsa, ctypes.c_void_p(mask.data_ptr()),
                                  ctypes.c_void_p(norms.data_ptr() if norms is not None else 0),
                                  ctypes.c_void_p(_stream_ptr(stream)))
    if rc != _lib.OK:
        raise SparseOITError(rc, "activeness launch failed")
    return mask, norms
