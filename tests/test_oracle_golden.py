"""The FP64 oracle against its frozen regression fixture (tests/golden/oracle_small.txt).

The fixture is not a pin to the paper (the paper prints no worked example);
it guards the pinned oracle against unnoticed changes to its arithmetic."""
import os

import numpy as np

from tests.golden.make_oracle_golden import OUT, compute


def test_oracle_matches_regression_fixture():
    want = [line.split() for line in open(OUT) if not line.startswith("#")]
    got = compute()
    assert len(got) == len(want)
    for (k, a, b, c, v), w in zip(got, want):
        assert (k, str(a), str(b), str(c)) == tuple(w[:4])
        ref = float(w[4])
        assert abs(v - ref) <= 1e-12 * max(1.0, abs(ref)), (k, a, b, c, v, ref)


def test_fixture_is_not_degenerate():
    want = [line.split() for line in open(OUT) if not line.startswith("#")]
    img = np.array([float(w[4]) for w in want if w[0] == "image_active"])
    grads = np.array([float(w[4]) for w in want if w[0] == "grad"])
    assert np.mean(~np.isin(img, (0.1, 0.2, 0.3))) > 0.5   # most sampled pixels see a splat
    assert np.mean(grads != 0.0) > 0.5
    assert os.path.getsize(OUT) < 64 * 1024
