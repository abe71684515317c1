"""FP64 oracle of the periodic active-set update (Sec. 4.1, Eq. 8).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain numpy, written
from the definitions:

* camera_centre: the pinhole camera x_cam = R x_world + t has its centre
  where x_cam = 0, c = -R^T t.
* fps_views: farthest point sampling over the training views' camera
  centres with a given first view (Sec. 4.1, "Updating Active Set via
  Subsampling"): repeatedly take the view farthest from its nearest already
  chosen view; ties go to the lowest index.
* group_norms / activeness: Eq. 8 with the quantifier read as "some
  attribute" (the sentence after Eq. 8): a splat is active when the
  Euclidean norm of at least one attribute group's gradient -- mu (3),
  q (4), log s (3), opacity logit (1), colour SH (48), weight SH (16) --
  is strictly above that group's threshold.
"""
import numpy as np

# columns of a 75-wide gradient row per attribute group (the oracle's row layout)
GROUP_COLUMNS = ((0, 3), (3, 7), (7, 10), (10, 11), (11, 59), (59, 75))


def camera_centre(cam) -> np.ndarray:
    R = np.asarray(cam["R"], dtype=np.float64).reshape(3, 3)
    t = np.asarray(cam["t"], dtype=np.float64).reshape(3)
    return -(R.T @ t)


def fps_views(cams, n_sub: int, first: int) -> list:
    c = np.stack([camera_centre(cm) for cm in cams])
    n = c.shape[0]
    if not (1 <= n_sub <= n and 0 <= first < n):
        raise ValueError("need 1 <= n_sub <= n and 0 <= first < n")
    chosen = [int(first)]
    nearest = np.full(n, np.inf)
    while len(chosen) < n_sub:
        last = c[chosen[-1]]
        d = ((c - last) ** 2).sum(axis=1)
        nearest = np.minimum(nearest, d)
        chosen.append(int(np.argmax(nearest)))  # argmax returns the lowest index among ties
    return chosen


def group_norms(grads: np.ndarray) -> np.ndarray:
    """[N, 75] gradient rows -> [N, 6] Euclidean norms per attribute group."""
    g = np.asarray(grads, dtype=np.float64)
    return np.stack([np.sqrt((g[:, a:b] ** 2).sum(axis=1)) for a, b in GROUP_COLUMNS], axis=1)


def activeness(grads: np.ndarray, eps) -> np.ndarray:
    """Eq. 8 (some-attribute reading): uint8 [N], 1 where some group's norm > eps of that group."""
    return (group_norms(grads) > np.asarray(eps, dtype=np.float64)[None, :]).any(axis=1).astype(np.uint8)
