"""Writes tests/golden/oracle_small.txt: a regression fixture of the FP64 oracle.

The paper prints no worked numeric example (its tables report image-quality
metrics and timings on real datasets), so no fixture in this folder holds
values from the paper.  This one freezes the oracle's own output on a small
seeded scene (64 splats of log-scale mean -1.5, one 32x32 view, half of the splats active): 48
sampled image values (full render, and active set over the complement's
sums) and 60 sampled gradient entries of the linear loss L = sum g.C, plus
dL/dsigma.  It calls only ``oracle`` and the seeded case generators; a
change to the oracle's arithmetic that moves any value shows up here, and a
regeneration names the passage that justifies it in its commit message.

Usage: python tests/golden/make_oracle_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from tests.oracle_cases import front_camera, small_random_scene  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_small.txt")


def case():
    scene = small_random_scene(64, 9001, log_scale_mean=-1.5)
    cam = front_camera(32, 32)
    rng = np.random.Generator(np.random.PCG64(9002))
    active = rng.random(64) < 0.5
    g = rng.normal(size=(32, 32, 3))
    pix = rng.integers(0, 32, size=(48, 2))
    ent = np.stack([rng.choice(np.where(active)[0], 60), rng.integers(0, 75, 60)], axis=1)
    return scene, cam, active, g, pix, ent


def compute():
    scene, cam, active, g, pix, ent = case()
    full = oracle.render(scene, cam)
    frozen, _, _ = oracle.render_sums(scene, cam, subset=~active)
    act = oracle.render(scene, cam, subset=active, frozen_sums=frozen)
    grads, dsig, _ = oracle.backward(scene, cam, act["sums"], g, active=active)
    rows = []
    for (y, x) in pix:
        for ch in range(3):
            rows.append(("image_full", int(y), int(x), ch, float(full["image"][y, x, ch])))
            rows.append(("image_active", int(y), int(x), ch, float(act["image"][y, x, ch])))
    for (i, j) in ent:
        rows.append(("grad", int(i), int(j), 0, float(grads[i, j])))
    rows.append(("dsigma", 0, 0, 0, float(dsig)))
    return rows


def main():
    rows = compute()
    with open(OUT, "w") as f:
        f.write("# FP64 oracle regression fixture; written by make_oracle_golden.py (calls only oracle/).\n")
        f.write("# kind a b c value   (image: y x channel; grad: splat column 0; dsigma: 0 0 0)\n")
        for k, a, b, c, v in rows:
            f.write(f"{k} {a} {b} {c} {v!r}\n")
    print(f"wrote {len(rows)} values to {OUT}")


if __name__ == "__main__":
    main()
