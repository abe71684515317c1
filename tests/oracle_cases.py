"""Hand-built scenes for the oracle's closed-form pins (no method arithmetic)."""
import numpy as np


def axis_camera(width=32, height=32, f=100.0):
    """Camera at the origin looking down +z; the optical axis hits the centre
    of pixel (width//2, height//2)."""
    return dict(R=np.eye(3, dtype=np.float32), t=np.zeros(3, dtype=np.float32), fx=f, fy=f,
                cx=width // 2 + 0.5, cy=height // 2 + 0.5, width=width, height=height)


def make_scene(means, log_scales=None, opacity_logits=None, quats=None, sh_color=None, sh_weight=None,
               sigma=6.0, bg=(0.0, 0.0, 0.0)):
    means = np.asarray(means, dtype=np.float64).reshape(-1, 3)
    n = means.shape[0]
    if quats is None:
        quats = np.tile([1.0, 0.0, 0.0, 0.0], (n, 1))
    if log_scales is None:
        log_scales = np.full((n, 3), -3.0)
    if opacity_logits is None:
        opacity_logits = np.zeros(n)
    if sh_color is None:
        sh_color = np.zeros((n, 16, 3))
    if sh_weight is None:
        sh_weight = np.zeros((n, 16))
    return dict(means=means, quats=np.asarray(quats, float).reshape(n, 4),
                log_scales=np.asarray(log_scales, float).reshape(n, 3),
                opacity_logits=np.asarray(opacity_logits, float).reshape(n),
                sh_color=np.asarray(sh_color, float).reshape(n, 16, 3),
                sh_weight=np.asarray(sh_weight, float).reshape(n, 16), sigma=float(sigma),
                bg=np.asarray(bg, float))


def logit(p):
    return float(np.log(p / (1.0 - p)))


def small_random_scene(n, seed, spread=0.6, log_scale_mean=-2.2):
    """A few splats in front of a 4-unit-away camera, sized to cover a 32x32 view."""
    rng = np.random.Generator(np.random.PCG64(seed))
    means = rng.uniform(-spread, spread, size=(n, 3))
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    ls = rng.normal(log_scale_mean, 0.4, size=(n, 3))
    ol = rng.normal(0.0, 1.0, size=n)
    sh = rng.normal(0.0, 0.05, size=(n, 16, 3))
    sh[:, 0, :] = rng.normal(0.0, 0.3, size=(n, 3))
    shw = rng.normal(0.0, 0.05, size=(n, 16))
    shw[:, 0] = rng.normal(0.0, 0.3, size=n)
    return make_scene(means, ls, ol, q, sh, shw, sigma=6.0, bg=(0.1, 0.2, 0.3))


def front_camera(width=32, height=32, dist=4.0, fov_deg=50.0, tilt=(0.3, -0.2)):
    """A camera at distance `dist` looking roughly at the origin (slightly tilted)."""
    pos = np.array([tilt[0], tilt[1], -dist])
    fwd = -pos / np.linalg.norm(pos)
    up = np.array([0.0, -1.0, 0.0])
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])
    t = -R @ pos
    f = (width / 2.0) / np.tan(np.radians(fov_deg) / 2.0)
    return dict(R=R, t=t, fx=f, fy=f * 1.05, cx=width / 2.0 + 0.3, cy=height / 2.0 - 0.2, width=width,
                height=height)
