"""Seeded synthetic scenes, cameras and active sets.

The paper trains on Mip-NeRF 360, Tanks & Temples and DeepBlending
(Sec. 5.1); none of them is available here, so these generators stand in for
them with the shapes, sizes and value distributions of the five workloads
the library is measured on.  This module holds input generation only (random
numbers and camera placement) and none of the renderer's arithmetic; it is
the one module that both the CUDA path's tests and the FP64 oracle read.

Every array is float32 (the library's input type); the oracle reads the same
float32 values widened to float64.

Splat attributes (all workloads): log-scales N(-3.5, 0.4) per axis;
quaternions normalised N(0, 1)^4 (w, x, y, z); opacity logits N(0, 1)
(opacity sigmoid(N(0,1))); colour SH [16, 3] with the DC band N(0, 0.3) and
bands 1-3 N(0, 0.05); the OIT-weight SH [16] drawn the same way (Sec. 5.1:
single channel, degree 3); sigma = 6 (Eq. 1); background c0 = 0 (Eq. 7).

Cameras: pinhole, 50 degree horizontal field of view, principal point at
the image centre, on the radius-4 sphere with |cos(polar angle)| <= 0.9,
looking at the origin with +z up; world -> camera rotation in OpenCV axes
(x right, y down, z forward).
"""
from __future__ import annotations

import math

import numpy as np

SIGMA = 6.0
FOV_DEG = 50.0
CAM_RADIUS = 4.0


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def look_at_camera(pos, width: int, height: int, fov_deg: float = FOV_DEG) -> dict:
    """Pinhole camera at `pos` looking at the origin, +z world up."""
    pos = np.asarray(pos, dtype=np.float64)
    fwd = -pos / np.linalg.norm(pos)
    up = np.array([0.0, 0.0, 1.0])
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd]).astype(np.float32)
    t = (-R.astype(np.float64) @ pos).astype(np.float32)
    f = (width / 2.0) / math.tan(math.radians(fov_deg) / 2.0)
    return dict(R=R, t=t, fx=np.float32(f), fy=np.float32(f), cx=np.float32(width / 2.0),
                cy=np.float32(height / 2.0), width=int(width), height=int(height))


def random_camera(seed: int, width: int, height: int) -> dict:
    rng = _rng(seed)
    while True:
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        if abs(d[2]) <= 0.9:
            return look_at_camera(CAM_RADIUS * d, width, height)


def _attributes(rng: np.random.Generator, n: int) -> dict:
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    log_scales = rng.normal(-3.5, 0.4, size=(n, 3))
    opacity_logits = rng.normal(0.0, 1.0, size=n)
    sh = rng.normal(0.0, 0.05, size=(n, 16, 3))
    sh[:, 0, :] = rng.normal(0.0, 0.3, size=(n, 3))
    shw = rng.normal(0.0, 0.05, size=(n, 16))
    shw[:, 0] = rng.normal(0.0, 0.3, size=n)
    return dict(quats=q.astype(np.float32), log_scales=log_scales.astype(np.float32),
                opacity_logits=opacity_logits.astype(np.float32), sh_color=sh.astype(np.float32),
                sh_weight=shw.astype(np.float32))


def _scene(means: np.ndarray, attrs: dict) -> dict:
    s = dict(means=np.ascontiguousarray(means, dtype=np.float32))
    s.update(attrs)
    s["sigma"] = np.float32(SIGMA)
    s["bg"] = np.zeros(3, dtype=np.float32)
    return s


def _uniform_ball(rng, n, radius):
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = radius * rng.uniform(size=n) ** (1.0 / 3.0)
    return d * r[:, None]


def uniform_cube_scene(n: int, seed: int) -> dict:
    """Means uniform in [-1, 1]^3 (the 4,096-splat tiny workload)."""
    rng = _rng(seed)
    means = rng.uniform(-1.0, 1.0, size=(n, 3))
    return _scene(means, _attributes(rng, n))


def clustered_scene(n: int, seed: int, blobs: int = 32) -> dict:
    """Mixture of `blobs` anisotropic normal blobs inside the unit ball.

    Blob centres uniform in the radius-0.6 ball, covariance R diag(a^2) R^T
    with a ~ U(0.05, 0.3) per axis and R a random rotation; points outside
    radius 1 are redrawn from their blob."""
    rng = _rng(seed)
    per = [n // blobs + (1 if b < n % blobs else 0) for b in range(blobs)]
    centres = _uniform_ball(rng, blobs, 0.6)
    out = []
    for b in range(blobs):
        q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        a = rng.uniform(0.05, 0.3, size=3)
        L = q * a[None, :]
        pts = np.zeros((0, 3))
        while pts.shape[0] < per[b]:
            cand = centres[b] + rng.normal(size=(per[b], 3)) @ L.T
            cand = cand[np.linalg.norm(cand, axis=1) <= 1.0]
            pts = np.concatenate([pts, cand])[: per[b]]
        out.append(pts)
    means = np.concatenate(out)
    return _scene(means, _attributes(rng, n))


def unbounded_scene(n: int, seed: int) -> dict:
    """70 % uniform in the radius-2 ball, 30 % at radius exp(U[ln 2, ln 50])."""
    rng = _rng(seed)
    n_in = int(round(0.7 * n))
    inner = _uniform_ball(rng, n_in, 2.0)
    d = rng.normal(size=(n - n_in, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = np.exp(rng.uniform(math.log(2.0), math.log(50.0), size=n - n_in))
    means = np.concatenate([inner, d * r[:, None]])
    perm = rng.permutation(n)
    return _scene(means[perm], _attributes(rng, n))


def random_active_mask(n: int, fraction: float, seed: int) -> np.ndarray:
    """Seeded uniform random subset of round(fraction * n) splats (uint8 mask)."""
    rng = _rng(seed)
    k = int(round(fraction * n))
    m = np.zeros(n, dtype=np.uint8)
    m[rng.choice(n, size=k, replace=False)] = 1
    return m


def proxy_active_mask(means: np.ndarray, fraction: float, seed: int) -> np.ndarray:
    """Active set from a seeded per-splat gradient-magnitude proxy.

    g_i = |N(0,1)| (1 + 4 [mu_i within 0.5 of one of 8 centres drawn uniformly
    in the radius-2 ball]); the ceil(fraction N) largest g are active, ties
    broken toward the lower index.  Spatially clustered, like the small,
    hard-to-fit objects the active set concentrates on (Sec. 1)."""
    n = means.shape[0]
    rng = _rng(seed)
    centres = _uniform_ball(rng, 8, 2.0)
    g = np.abs(rng.normal(size=n))
    near = np.zeros(n, dtype=bool)
    for c in centres:
        near |= np.linalg.norm(means.astype(np.float64) - c, axis=1) <= 0.5
    g = g * (1.0 + 4.0 * near)
    k = int(math.ceil(fraction * n))
    order = np.lexsort((np.arange(n), -g))
    m = np.zeros(n, dtype=np.uint8)
    m[order[:k]] = 1
    return m


def uniform_target(seed: int, width: int, height: int) -> np.ndarray:
    return _rng(seed).uniform(0.0, 1.0, size=(height, width, 3)).astype(np.float32)


# Workloads (sizes of the five measured configurations).
TINY = dict(n=4096, width=128, height=128, seed=1000)
CLUSTERED = dict(n=200_000, width=800, height=800, seed=2000, active=0.10)
UNBOUNDED = dict(n=1_000_000, width=1297, height=840, seed=3000, fractions=(0.01, 0.05, 0.20, 1.0))
BATCHED = dict(n=3_000_000, seed=4000, active=0.05,
               resolutions=((640, 480), (800, 800), (1297, 840), (1600, 1064)), views_per_res=4)
PRECISION = dict(n=3_000_000, seed=5000, active=0.05, width=1297, height=840, views=8,
                 crop=(520, 292, 776, 548))
# periodic active-set update: the unbounded scene seen from 60 training views, 30 picked by
# farthest point sampling from a seeded first view (the paper's S = 30)
ACTIVE_UPDATE = dict(n=1_000_000, seed=3000, width=1297, height=840, views=60, n_sub=30, camera_seed=6000)


def tiny_workload():
    c = TINY
    scene = uniform_cube_scene(c["n"], c["seed"])
    target_scene = uniform_cube_scene(c["n"], c["seed"] + 1)
    cam = random_camera(c["seed"] + 3, c["width"], c["height"])
    return scene, target_scene, cam


def clustered_workload():
    c = CLUSTERED
    scene = clustered_scene(c["n"], c["seed"])
    mask = random_active_mask(c["n"], c["active"], c["seed"] + 2)
    cam = random_camera(c["seed"] + 3, c["width"], c["height"])
    target = uniform_target(c["seed"] + 1, c["width"], c["height"])
    return scene, mask, cam, target


def unbounded_workload(n: int | None = None, width: int | None = None, height: int | None = None):
    c = UNBOUNDED
    n = c["n"] if n is None else n
    W = c["width"] if width is None else width
    H = c["height"] if height is None else height
    scene = unbounded_scene(n, c["seed"])
    cam = random_camera(c["seed"] + 3, W, H)
    target = uniform_target(c["seed"] + 1, W, H)
    return scene, cam, target


def unbounded_active_mask(scene: dict, fraction: float) -> np.ndarray:
    return proxy_active_mask(scene["means"], fraction, UNBOUNDED["seed"] + 2)


def batched_cameras(seed: int = BATCHED["seed"]):
    cams = []
    k = 0
    for (W, H) in BATCHED["resolutions"]:
        for _ in range(BATCHED["views_per_res"]):
            cams.append(random_camera(seed + 3 + 17 * k, W, H))
            k += 1
    return cams


def precision_cameras(seed: int = PRECISION["seed"]):
    return [random_camera(seed + 3 + 17 * k, PRECISION["width"], PRECISION["height"])
            for k in range(PRECISION["views"])]


def training_cameras(n_views: int, seed: int, width: int, height: int) -> list:
    """n_views cameras drawn by the common camera rule, one seed each."""
    return [random_camera(seed + k, width, height) for k in range(n_views)]
