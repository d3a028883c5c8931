"""Writes tests/golden/config0_oracle_digest.json: a digest of the CPU FP64
oracle's render of the seeded config-0 scene (2k Gaussians in front of and
behind a textured quad, 128x128).  It calls only the oracle and the seeded
scene generator; the test-suite re-renders and compares, so any change to the
oracle's arithmetic shows up as a diff here and must be justified.

The paper prints no worked numeric example (no per-pixel value, image or
table entry that a renderer could reproduce), so this file pins the oracle to
its own committed state, not to the paper; the pins against the paper's
equations are the closed-form tests in test_oracle_pins.py.

Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O                      # noqa: E402
from paper_2506_06988_b300 import scenes           # noqa: E402


def digest(seed=1):
    s = scenes.config0_scene(seed)
    r = O.render(s)
    o = r.out
    return {
        "scene": f"config0 seed {seed}",
        "rgb_sum": [float(v) for v in o.rgb.sum(1)],
        "T_sum": float(o.T.sum()),
        "n_contrib_sum": int(o.n_contrib.sum()),
        "n_contrib_hist": np.bincount(o.n_contrib, minlength=32)[:32].tolist(),
        "evaluated_sum": int(o.evaluated.sum()),
        "tri_hits": np.bincount(r.mesh.tri_id + 1, minlength=3).tolist(),
        "mesh_depth_sum": float(r.mesh.depth.astype(np.float64).sum()),
        "ambiguous_pixels": int(o.amb.sum()),
        "pixel_4242_rgb": [float(v) for v in o.rgb[:, 4242]],
        "pixel_4242_T": float(o.T[4242]),
    }


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config0_oracle_digest.json")
    with open(out, "w") as f:
        json.dump(digest(), f, indent=1)
    print("wrote", out)
