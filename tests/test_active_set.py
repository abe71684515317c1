"""Active-set update (Sec. 4.1, Eq. 8): the oracle's view subsampling and
activeness test against closed forms, and the library's host-side view
subsampling against the oracle (no GPU needed)."""
import numpy as np
import pytest

import oracle
from oracle import active_set as oas
from paper_2605_13855_gb300 import scenes


def _cam_at(c):
    """A camera whose centre is c (R = I, t = -c)."""
    c = np.asarray(c, dtype=np.float64)
    return dict(R=np.eye(3, dtype=np.float32), t=(-c).astype(np.float32), fx=100.0, fy=100.0, cx=16.0, cy=16.0,
                width=32, height=32)


def test_camera_centre_of_look_at_camera():
    cam = scenes.look_at_camera(np.array([1.0, -2.0, 3.0]), 64, 48)
    assert np.allclose(oas.camera_centre(cam), [1.0, -2.0, 3.0], atol=1e-6)


def test_fps_square_ring_closed_form():
    # the 8 points of a 3x3 grid around its centre (exact squared distances):
    # from corner 0 the opposite corner 7; then the other two corners tie at
    # squared distance 4 (lower index 2 first, then 5); then every edge
    # midpoint is at distance 1 from a chosen corner (tie: lowest index, 1)
    pts = [(-1, -1), (0, -1), (1, -1), (-1, 0), (1, 0), (-1, 1), (0, 1), (1, 1)]
    cams = [_cam_at([2.0 * x, 2.0 * y, 3.0]) for x, y in pts]
    assert oas.fps_views(cams, 5, 0) == [0, 7, 2, 5, 1]
    assert oas.fps_views(cams, 2, 4) == [4, 0]


def test_fps_points_on_a_line():
    xs = [0.0, 1.0, 2.0, 10.0, 4.5]
    cams = [_cam_at([x, 0.0, 0.0]) for x in xs]
    # from 0: 10 (index 3); then the point farthest from {0, 10}: 4.5 (index 4, distance 4.5 vs 2 for x = 2)
    assert oas.fps_views(cams, 4, 0) == [0, 3, 4, 2]


def test_fps_is_invariant_under_rigid_motion():
    rng = np.random.default_rng(3)
    c = rng.normal(size=(40, 3)) * 3
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    moved = c @ q.T + np.array([5.0, -1.0, 2.0])
    a = oas.fps_views([_cam_at(x) for x in c], 10, 7)
    b = oas.fps_views([_cam_at(x) for x in moved], 10, 7)
    assert a == b and len(set(a)) == 10


def test_group_norms_and_activeness_closed_form():
    g = np.zeros((4, 75))
    g[0, 0:3] = [3.0, 4.0, 0.0]        # |mu| = 5
    g[1, 10] = -2.0                    # |opacity| = 2
    g[2, 11:59] = 0.5                  # |h| = 0.5 sqrt(48)
    g[3, 59:75] = 1.0                  # |w| = 4
    n = oas.group_norms(g)
    assert np.allclose(n[0], [5, 0, 0, 0, 0, 0]) and np.allclose(n[1], [0, 0, 0, 2, 0, 0])
    assert np.isclose(n[2, 4], 0.5 * np.sqrt(48)) and np.isclose(n[3, 5], 4.0)
    eps = [5.0, 1.0, 1.0, 1.9, 10.0, 3.9]
    # strict inequality (|mu| = 5 is not above 5); one active group suffices (row 1, 3)
    assert list(oas.activeness(g, eps)) == [0, 1, 0, 1]
    # a row whose groups are all below their thresholds stays inactive even when their sum is not
    g2 = np.zeros((1, 75))
    g2[0, 0] = 0.9
    g2[0, 3] = 0.9
    assert oas.activeness(g2, [1.0] * 6)[0] == 0


def test_library_fps_matches_oracle():
    from paper_2605_13855_gb300 import renderer
    for seed in range(5):
        cams = [scenes.random_camera(1000 * seed + k, 64, 48) for k in range(25)]
        first = seed % 25
        assert renderer.fps_views(cams, 12, first) == oas.fps_views(cams, 12, first)
    pts = [(-1, -1), (0, -1), (1, -1), (-1, 0), (1, 0), (-1, 1), (0, 1), (1, 1)]
    ring = [_cam_at([2.0 * x, 2.0 * y, 3.0]) for x, y in pts]
    assert renderer.fps_views(ring, 5, 0) == [0, 7, 2, 5, 1]  # the tie rule
    with pytest.raises(Exception):
        renderer.fps_views(cams, 26, 0)
    with pytest.raises(Exception):
        renderer.fps_views(cams, 3, 25)
