"""Pins of the FP64 oracle against things other than itself (CPU only).

* SH basis: SciPy's complex spherical harmonics, orthonormality by
  quadrature, the zonal values sqrt((2l+1)/4pi) at the pole, and finite
  differences of its polynomial gradient.
* Eq. 2 / 6: the 2D covariance equals J_fd Sigma J_fd^T + 0.3 I with Sigma
  built from SciPy's quaternion rotation and J_fd a finite-difference
  Jacobian of the oracle's own projected centre.
* Eq. 5 / 7: closed forms for one and two splats on the optical axis.
* Binning: the bbox-binned render is bit-identical to the brute-force one.
* Order independence (Sec. A: blending independent of depth order) and the
  active / frozen identity (Sec. 4.1).
* Eq. 10 chained to all parameters: central finite differences of the
  oracle's own forward pass.
"""
import math

import numpy as np
import pytest

import oracle
from tests.oracle_cases import axis_camera, front_camera, logit, make_scene, small_random_scene


# ------------------------------------------------------------------ SH ----

def _real_sh_scipy(l, m, n):
    from scipy.special import sph_harm_y
    x, y, z = n
    theta = math.acos(max(-1.0, min(1.0, z)))
    phi = math.atan2(y, x)
    if m == 0:
        return float(np.real(sph_harm_y(l, 0, theta, phi)))
    Y = sph_harm_y(l, abs(m), theta, phi)
    # SciPy includes the Condon-Shortley phase (-1)^m; the oracle's basis does not.
    s = math.sqrt(2.0) * (-1.0) ** abs(m)
    return float(s * (np.real(Y) if m > 0 else np.imag(Y)))


def test_sh_matches_scipy():
    rng = np.random.default_rng(0)
    for _ in range(50):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        Y, _ = oracle.sh_basis(n)
        for l in range(4):
            for m in range(-l, l + 1):
                assert Y[l * l + l + m] == pytest.approx(_real_sh_scipy(l, m, n), abs=1e-13)


def test_sh_zonal_values_at_pole():
    Y, _ = oracle.sh_basis([0.0, 0.0, 1.0])
    for l in range(4):
        for m in range(-l, l + 1):
            want = math.sqrt((2 * l + 1) / (4 * math.pi)) if m == 0 else 0.0
            assert Y[l * l + l + m] == pytest.approx(want, abs=1e-15)
    assert Y[0] == pytest.approx(1.0 / (2.0 * math.sqrt(math.pi)), abs=1e-16)


def test_sh_orthonormal_by_quadrature():
    # Gauss-Legendre in cos(theta) x uniform phi is exact for these degrees.
    xs, ws = np.polynomial.legendre.leggauss(12)
    nphi = 16
    G = np.zeros((16, 16))
    for z, wz in zip(xs, ws):
        r = math.sqrt(1.0 - z * z)
        for k in range(nphi):
            phi = 2.0 * math.pi * k / nphi
            Y, _ = oracle.sh_basis([r * math.cos(phi), r * math.sin(phi), z])
            G += wz * (2.0 * math.pi / nphi) * np.outer(Y, Y)
    assert np.abs(G - np.eye(16)).max() < 1e-13


def test_sh_gradient_finite_difference():
    rng = np.random.default_rng(1)
    h = 1e-6
    for _ in range(10):
        n = rng.normal(size=3)
        _, dY = oracle.sh_basis(n)
        for e in range(3):
            dp = n.copy(); dp[e] += h
            dm = n.copy(); dm[e] -= h
            fd = (oracle.sh_basis(dp)[0] - oracle.sh_basis(dm)[0]) / (2 * h)
            assert np.abs(fd - dY[:, e]).max() < 1e-8


# ------------------------------------------------------- projection ------

def test_cov2d_matches_fd_jacobian_and_scipy_rotation():
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(2)
    cam = front_camera(64, 48)
    for _ in range(20):
        mu = rng.uniform(-0.8, 0.8, size=3)
        q = rng.normal(size=4)
        ls = rng.normal(-2.5, 0.5, size=3)
        sc = make_scene([mu], [ls], [2.0], [q])
        pr = oracle.project(sc, cam)[0]
        assert pr[0] == 1.0
        # Sigma from SciPy's rotation (scalar-last quaternion convention)
        Rq = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        Sig = Rq @ np.diag(np.exp(2 * ls)) @ Rq.T
        # Jacobian of the projected centre w.r.t. the world mean, by central FD
        Jw = np.zeros((2, 3))
        h = 1e-6
        for e in range(3):
            mp = mu.copy(); mp[e] += h
            mm = mu.copy(); mm[e] -= h
            pp = oracle.project(make_scene([mp], [ls], [2.0], [q]), cam)[0]
            pm = oracle.project(make_scene([mm], [ls], [2.0], [q]), cam)[0]
            Jw[:, e] = (pp[1:3] - pm[1:3]) / (2 * h)
        C = Jw @ Sig @ Jw.T + 0.3 * np.eye(2)
        got = np.array([[pr[3], pr[4]], [pr[4], pr[5]]])
        assert np.abs(got - C).max() < 1e-6 * max(1.0, np.abs(C).max())
        # conic is the inverse
        K = np.array([[pr[6], pr[7]], [pr[7], pr[8]]])
        assert np.abs(K @ got - np.eye(2)).max() < 1e-10


# ------------------------------------------------------ closed forms -----

def _zonal(l):
    return math.sqrt((2 * l + 1) / (4 * math.pi))


def test_single_splat_on_axis_closed_form():
    cam = axis_camera(33, 33, f=100.0)
    z, o, s = 3.0, 0.7, math.exp(-3.0)
    sh = np.zeros((16, 3))
    sh[0] = [0.4, -0.2, 0.1]       # l=0
    sh[2] = [0.1, 0.05, -0.3]      # l=1, m=0
    sh[12] = [0.02, 0.0, 0.05]     # l=3, m=0
    sh[5] = [9.0, 9.0, 9.0]        # l=2, m=-1: zero at the pole
    shw = np.zeros(16)
    shw[0] = 0.3
    shw[6] = -0.1                  # l=2, m=0
    bg = (0.2, 0.4, 0.6)
    sc = make_scene([[0, 0, z]], [[math.log(s)] * 3], [logit(o)], sh_color=[sh], sh_weight=[shw],
                    sigma=6.0, bg=bg)
    r = oracle.render(sc, cam)
    c = 0.5 + sh[0] * _zonal(0) + sh[2] * _zonal(1) + sh[12] * _zonal(3)
    v = 0.5 + shw[0] * _zonal(0) + shw[6] * _zonal(2)
    w = (1.0 - z / 6.0) * v
    var = (cam["fx"] * s / z) ** 2 + 0.3     # Eq. 6 on the axis + dilation
    for k in range(0, 6):
        a = o * math.exp(-0.5 * k * k / var)
        if a < 1 / 255:
            continue
        want = (1 - a) * np.array(bg) + a * c
        assert np.allclose(r["image"][16, 16 + k], want, atol=1e-14, rtol=0)
        assert r["sums"][3, 16, 16 + k] == pytest.approx(a * w, rel=1e-14)
        assert r["sums"][4, 16, 16 + k] == pytest.approx(math.log(1 - a), rel=1e-13)


def test_two_splats_weighted_average():
    cam = axis_camera(17, 17, f=100.0)
    o1, o2 = 0.6, 0.3
    sh = np.zeros((2, 16, 3))
    sh[0, 0] = [0.5, 0.0, -0.5]
    sh[1, 0] = [-0.3, 0.6, 0.2]
    shw = np.zeros((2, 16))
    shw[0, 0] = 0.2
    shw[1, 0] = -0.4
    z = np.array([2.0, 4.0])
    sc = make_scene([[0, 0, z[0]], [0, 0, z[1]]], None, [logit(o1), logit(o2)], sh_color=sh, sh_weight=shw,
                    sigma=5.0, bg=(0.3, 0.3, 0.3))
    img = oracle.render(sc, cam)["image"][8, 8]
    c = 0.5 + sh[:, 0, :] * _zonal(0)
    v = 0.5 + shw[:, 0] * _zonal(0)
    w = (1 - z / 5.0) * v
    a = np.array([o1, o2])
    T = (1 - a[0]) * (1 - a[1])
    F = (a[0] * w[0] * c[0] + a[1] * w[1] * c[1]) / (a[0] * w[0] + a[1] * w[1])
    assert np.allclose(img, T * 0.3 + (1 - T) * F, atol=1e-14, rtol=0)
    # listing the splats in the other order leaves the image unchanged (order independence)
    img2 = oracle.render(make_scene([[0, 0, z[1]], [0, 0, z[0]]], None, [logit(o2), logit(o1)],
                                    sh_color=sh[::-1].copy(), sh_weight=shw[::-1].copy(), sigma=5.0,
                                    bg=(0.3, 0.3, 0.3)), cam)["image"][8, 8]
    assert np.allclose(img2, img, atol=1e-15, rtol=0)


def test_view_direction_from_off_origin_camera():
    """Eq. 4: the SH argument is the unit vector from the camera centre to the mean.
    Camera on the sphere looking at a splat at the origin: n = the camera's forward axis."""
    pos = np.array([1.2, -2.5, 2.9])
    fwd = -pos / np.linalg.norm(pos)
    right = np.cross(fwd, [0.0, 0.0, 1.0]); right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])
    cam = dict(R=R, t=-R @ pos, fx=80.0, fy=80.0, cx=8.5, cy=8.5, width=17, height=17)
    sh = np.zeros((16, 3))
    sh[0] = [0.1, 0.0, 0.2]
    sh[1] = [0.3, -0.2, 0.1]   # l=1, m=-1 (y)
    sh[2] = [-0.1, 0.25, 0.0]  # l=1, m=0  (z)
    sh[3] = [0.2, 0.1, -0.3]   # l=1, m=1  (x)
    o = 0.8
    sc = make_scene([[0.0, 0.0, 0.0]], [[-2.0] * 3], [logit(o)], sh_color=[sh], sigma=9.0, bg=(0.0, 0.0, 0.0))
    img = oracle.render(sc, cam)["image"][8, 8]
    n = fwd
    k1 = math.sqrt(3.0 / (4.0 * math.pi))
    c = 0.5 + sh[0] * _zonal(0) + k1 * (n[1] * sh[1] + n[2] * sh[2] + n[0] * sh[3])
    assert np.allclose(img, o * c, atol=1e-14, rtol=0)


def test_far_splat_attenuates_only():
    """A splat beyond sigma has w = 0: Q = 0, F := 0 and C = T c0 (Eq. 1, 7)."""
    cam = axis_camera(9, 9, f=50.0)
    sc = make_scene([[0, 0, 7.0]], [[-1.0] * 3], [logit(0.5)], sigma=6.0, bg=(0.2, 0.4, 0.6))
    r = oracle.render(sc, cam)
    assert r["sums"][3, 4, 4] == 0.0
    assert np.allclose(r["image"][4, 4], 0.5 * np.array([0.2, 0.4, 0.6]), atol=1e-15, rtol=0)


def test_alpha_threshold_and_clamp():
    cam = axis_camera(9, 9, f=50.0)
    # opacity below 1/255 never contributes
    sc = make_scene([[0, 0, 2.0]], [[-1.0] * 3], [logit(0.9 / 255)], bg=(0.5, 0.5, 0.5))
    r = oracle.render(sc, cam)
    assert r["pairs"] == 0 and np.all(r["image"] == 0.5)
    # opacity 0.999 is clamped to 0.99 at the centre
    sc = make_scene([[0, 0, 2.0]], [[-1.0] * 3], [logit(0.999)], bg=(0.5, 0.5, 0.5))
    r = oracle.render(sc, cam)
    assert r["sums"][4, 4, 4] == pytest.approx(math.log(0.01), rel=1e-13)
    assert r["clamped"] >= 1


# ----------------------------------------------- binning / invariants ----

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_binned_equals_brute_force_bitwise(seed):
    sc = small_random_scene(200, seed)
    cam = front_camera(64, 40)
    a, amb_a, st_a = oracle.render_sums(sc, cam, brute=True, amb_band=1e-3, want_amb=True)
    b, amb_b, st_b = oracle.render_sums(sc, cam, brute=False, amb_band=1e-3, want_amb=True)
    assert st_a == st_b and st_a[0] > 1000
    assert np.array_equal(a, b)
    assert np.array_equal(amb_a, amb_b)
    # a window and a subset as well
    m = (np.arange(200) % 3 == 0)
    a, _, _ = oracle.render_sums(sc, cam, subset=m, brute=True, window=(5, 7, 50, 33))
    b, _, _ = oracle.render_sums(sc, cam, subset=m, brute=False, window=(5, 7, 50, 33))
    assert np.array_equal(a, b)
    full, _, _ = oracle.render_sums(sc, cam, subset=m)
    assert np.array_equal(b[:, 7:33, 5:50], full[:, 7:33, 5:50])
    assert np.all(b[:, :7] == 0) and np.all(b[:, :, 50:] == 0)


def test_permutation_invariance():
    sc = small_random_scene(300, 5)
    cam = front_camera(48, 48)
    perm = np.random.default_rng(7).permutation(300)
    sc2 = {k: (v[perm] if isinstance(v, np.ndarray) and v.ndim >= 1 and v.shape[0] == 300 else v)
           for k, v in sc.items()}
    a = oracle.render(sc, cam)["image"]
    b = oracle.render(sc2, cam)["image"]
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


@pytest.mark.parametrize("frac", [0.0, 0.3, 1.0])
def test_active_plus_frozen_equals_full(frac):
    sc = small_random_scene(250, 11)
    cam = front_camera(48, 40)
    rng = np.random.default_rng(3)
    act = rng.uniform(size=250) < frac
    full = oracle.render(sc, cam)
    frozen, _, _ = oracle.render_sums(sc, cam, subset=~act)
    part = oracle.render(sc, cam, subset=act, frozen_sums=frozen)
    assert np.abs(part["sums"] - full["sums"]).max() <= 1e-12 * max(1.0, np.abs(full["sums"]).max())
    assert np.abs(part["image"] - full["image"]).max() <= 1e-12
    # gradients of the active splats are those of the full render
    g = np.random.default_rng(4).normal(size=full["image"].shape)
    gf, sf, _ = oracle.backward(sc, cam, full["sums"], g)
    ga, sa, _ = oracle.backward(sc, cam, part["sums"], g, active=act)
    assert np.all(np.isnan(ga[~act]))
    if act.any():
        assert np.abs(ga[act] - gf[act]).max() <= 1e-10 * max(1.0, np.abs(gf).max())


# ------------------------------------------------- finite differences ----

GROUPS = dict(means=(0, 3), quats=(3, 7), log_scales=(7, 10), opacity_logits=(10, 11),
              sh_color=(11, 59), sh_weight=(59, 75))


def _set_param(sc, i, j, val):
    for name, (lo, hi) in GROUPS.items():
        if lo <= j < hi:
            arr = sc[name].reshape(sc[name].shape[0], -1)
            arr[i, j - lo] = val
            return
    raise IndexError(j)


def _get_param(sc, i, j):
    for name, (lo, hi) in GROUPS.items():
        if lo <= j < hi:
            return float(sc[name].reshape(sc[name].shape[0], -1)[i, j - lo])
    raise IndexError(j)


def _loss(sc, cam, g):
    return float(np.sum(oracle.render(sc, cam)["image"] * g))


@pytest.mark.parametrize("seed,opacity_shift", [(21, 0.0), (22, 0.0), (23, 9.0)])
def test_gradient_matches_central_finite_differences(seed, opacity_shift):
    sc = small_random_scene(40, seed, log_scale_mean=-2.0)
    sc["opacity_logits"] = sc["opacity_logits"] + opacity_shift  # shift 9: pairs clamped at 0.99
    for k in ("means", "quats", "log_scales", "opacity_logits", "sh_color", "sh_weight"):
        sc[k] = sc[k].copy()
    # with the shift, a narrow field of view makes splats ~6 px wide so that the
    # clamped core (p < ln(1/0.99), radius 0.14 sigma') covers whole pixels
    cam = front_camera(32, 28, fov_deg=12.0 if opacity_shift > 0 else 50.0)
    r = oracle.render(sc, cam)
    g = np.random.default_rng(seed).normal(size=r["image"].shape)
    grads, dsig, amb = oracle.backward(sc, cam, r["sums"], g, amb_band=1e-3)
    rng = np.random.default_rng(seed + 100)
    ok = np.where((amb == 0) & (oracle.project(sc, cam)[:, 0] == 1))[0]
    assert ok.size > 20
    checked = 0
    for i in rng.choice(ok, size=12, replace=False):
        for j in list(range(0, 11)) + list(rng.choice(np.arange(11, 75), size=8, replace=False)):
            x0 = _get_param(sc, i, j)
            h = 1e-6 * max(1.0, abs(x0))
            _set_param(sc, i, j, x0 + h)
            lp = _loss(sc, cam, g)
            _set_param(sc, i, j, x0 - h)
            lm = _loss(sc, cam, g)
            _set_param(sc, i, j, x0)
            fd = (lp - lm) / (2 * h)
            scale = max(1e-3, np.abs(grads[i]).max())
            assert abs(fd - grads[i, j]) <= 2e-6 * scale + 1e-7, (i, j, fd, grads[i, j])
            checked += 1
    assert checked > 200
    if opacity_shift > 0:
        assert r["clamped"] > 20
    # sigma (Eq. 1): every splat's weight depends on it
    proj = oracle.project(sc, cam)
    if np.all(np.abs(proj[proj[:, 0] == 1, 21]) > 1e-3):
        s0 = sc["sigma"]
        h = 1e-6 * s0
        sc["sigma"] = s0 + h
        lp = _loss(sc, cam, g)
        sc["sigma"] = s0 - h
        lm = _loss(sc, cam, g)
        sc["sigma"] = s0
        assert abs((lp - lm) / (2 * h) - dsig) <= 1e-6 * max(1.0, abs(dsig))


# ------------------------------------------- clamps and the near plane ----

def test_negative_colour_channel_is_clamped_to_zero():
    """Eq. 4 with the max(0, .) activation: a channel whose SH value is below zero renders as a
    zero colour, so a lone splat on the axis gives (1 - a) c0 in that channel and (1 - a) c0 + a c
    in the others; that channel's coefficients get no gradient."""
    cam = axis_camera(33, 33, f=100.0)
    z, o, s = 3.0, 0.7, math.exp(-3.0)
    sh = np.zeros((16, 3))
    sh[0] = [-2.5, 0.3, 0.0]        # red: 0.5 - 2.5 Y00 = -0.205 < 0
    shw = np.zeros(16)
    shw[0] = 0.3
    bg = (0.2, 0.4, 0.6)
    sc = make_scene([[0, 0, z]], [[math.log(s)] * 3], [logit(o)], sh_color=[sh], sh_weight=[shw],
                    sigma=6.0, bg=bg)
    r = oracle.render(sc, cam)
    c = 0.5 + sh[0] * _zonal(0)
    assert c[0] < -0.1
    c_act = np.maximum(c, 0.0)
    var = (cam["fx"] * s / z) ** 2 + 0.3
    for k in range(0, 6):
        a = o * math.exp(-0.5 * k * k / var)
        want = (1 - a) * np.array(bg) + a * c_act
        assert np.allclose(r["image"][16, 16 + k], want, atol=1e-14, rtol=0)
        assert r["sums"][0, 16, 16 + k] == 0.0
    # gradient of a linear loss on the red channel only: the red SH is dead, green is not
    g = np.zeros(r["image"].shape)
    g[..., 0] = 1.0
    g[..., 1] = 1.0
    grads, _, _ = oracle.backward(sc, cam, r["sums"], g)
    red = grads[0, 11:59].reshape(16, 3)[:, 0]
    green = grads[0, 11:59].reshape(16, 3)[:, 1]
    assert np.all(red == 0.0)
    assert abs(green[0]) > 1e-3


def test_negative_weight_sh_gives_zero_weight():
    """Eq. 1 with v = max(0, SH + 0.5): a splat whose weight SH is below zero has w = 0.  It still
    attenuates (T) but adds nothing to P or Q: alone it renders (1 - a) c0 (Q = 0, F := 0); beside a
    positive-weight splat the normalised colour is the other splat's colour exactly."""
    cam = axis_camera(17, 17, f=100.0)
    o1, o2 = 0.6, 0.3
    sh = np.zeros((2, 16, 3))
    sh[0, 0] = [0.5, 0.0, -0.5]
    sh[1, 0] = [-0.3, 0.6, 0.2]
    shw = np.zeros((2, 16))
    shw[0, 0] = -2.5                # v_raw = 0.5 - 2.5 Y00 < 0
    shw[1, 0] = 0.2
    bg = (0.3, 0.2, 0.1)
    z = np.array([2.0, 4.0])
    lone = make_scene([[0, 0, z[0]]], None, [logit(o1)], sh_color=sh[:1], sh_weight=shw[:1], sigma=5.0, bg=bg)
    r = oracle.render(lone, cam)
    assert r["sums"][3, 8, 8] == 0.0 and np.all(r["sums"][:3, 8, 8] == 0.0)
    assert np.allclose(r["image"][8, 8], (1 - o1) * np.array(bg), atol=1e-15, rtol=0)
    both = make_scene([[0, 0, z[0]], [0, 0, z[1]]], None, [logit(o1), logit(o2)], sh_color=sh, sh_weight=shw,
                      sigma=5.0, bg=bg)
    img = oracle.render(both, cam)["image"][8, 8]
    c2 = 0.5 + sh[1, 0] * _zonal(0)
    T = (1 - o1) * (1 - o2)
    assert np.allclose(img, T * np.array(bg) + (1 - T) * c2, atol=1e-14, rtol=0)
    # the clamped weight SH gets no gradient; the same splat with a positive weight does
    rb = oracle.render(both, cam)
    grads, _, _ = oracle.backward(both, cam, rb["sums"], np.ones(rb["image"].shape))
    assert np.all(grads[0, 59:75] == 0.0)
    live = make_scene([[0, 0, z[0]], [0, 0, z[1]]], None, [logit(o1), logit(o2)], sh_color=sh,
                      sh_weight=np.abs(shw) * 0.1, sigma=5.0, bg=bg)
    rl = oracle.render(live, cam)
    gl, _, _ = oracle.backward(live, cam, rl["sums"], np.ones(rl["image"].shape))
    assert abs(gl[0, 59]) > 1e-3


@pytest.mark.parametrize("tz,visible", [(0.19, False), (0.2, False), (0.21, True)])
def test_near_plane_cull_at_depth_point_two(tz, visible):
    """The near-plane cull drops a splat whose camera-space depth is at most 0.2 (3DGS convention):
    identical splats on the axis at t_z = 0.19 and 0.2 leave the view empty, at 0.21 it renders."""
    cam = axis_camera(33, 33, f=100.0)
    o, s = 0.7, math.exp(-3.0)
    sh = np.zeros((16, 3))
    sh[0] = [0.4, 0.2, 0.1]
    bg = (0.2, 0.4, 0.6)
    sc = make_scene([[0, 0, tz]], [[math.log(s)] * 3], [logit(o)], sh_color=[sh], sigma=6.0, bg=bg)
    r = oracle.render(sc, cam)
    pr = oracle.project(sc, cam)[0]
    if visible:
        assert pr[0] == 1.0 and r["pairs"] > 0
        c = 0.5 + sh[0] * _zonal(0)
        assert np.allclose(r["image"][16, 16], (1 - o) * np.array(bg) + o * c, atol=1e-14, rtol=0)
    else:
        assert pr[0] == 0.0 and r["pairs"] == 0
        assert np.all(r["image"] == np.array(bg))


def test_splat_beyond_sigma_gets_no_weight_gradient():
    """Eq. 1 with max(0, 1 - d/sigma): a splat deeper than sigma has w = 0 whatever its weight SH,
    so its weight SH, and sigma through it, get no gradient.  Beside two splats in front of sigma, the
    oracle's dL/dsigma equals a central finite difference (the far splat stays clamped under the
    perturbation) and the far splat's weight-SH gradient is exactly zero."""
    cam = axis_camera(17, 17, f=100.0)
    sh = np.zeros((3, 16, 3))
    sh[0, 0] = [0.5, 0.0, -0.5]
    sh[1, 0] = [-0.3, 0.6, 0.2]
    sh[2, 0] = [0.4, -0.4, 0.3]
    shw = np.zeros((3, 16))
    shw[0, 0] = 0.4
    shw[1, 0] = 0.2
    shw[2, 0] = -0.1
    sc = make_scene([[0, 0, 7.0], [0.01, 0, 2.0], [-0.02, 0.01, 3.0]], [[-1.0] * 3, [-1.5] * 3, [-1.2] * 3],
                    [logit(0.6), logit(0.5), logit(0.4)], sh_color=sh, sh_weight=shw, sigma=6.0,
                    bg=(0.3, 0.2, 0.1))
    r = oracle.render(sc, cam)
    g = np.random.default_rng(5).normal(size=r["image"].shape)
    grads, dsig, _ = oracle.backward(sc, cam, r["sums"], g)
    assert np.all(grads[0, 59:75] == 0.0)
    assert np.any(np.abs(grads[1, 59:75]) > 1e-6)
    h = 1e-6 * sc["sigma"]
    s0 = sc["sigma"]
    sc["sigma"] = s0 + h
    lp = float(np.sum(oracle.render(sc, cam)["image"] * g))
    sc["sigma"] = s0 - h
    lm = float(np.sum(oracle.render(sc, cam)["image"] * g))
    sc["sigma"] = s0
    fd = (lp - lm) / (2 * h)
    assert abs(fd) > 1e-6
    assert abs(fd - dsig) <= 1e-6 * max(1.0, abs(dsig))
