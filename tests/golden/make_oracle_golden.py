"""Writes oracle_small.json: the FP64 oracle's outputs on small seeded scenes.

Calls only ``oracle`` (and the seeded input generators); nothing here comes
from the CUDA path.  Run from the repository root:

    python tests/golden/make_oracle_golden.py

The fixture freezes the oracle: a later change to its arithmetic that moves
any value fails ``tests/test_golden.py`` until this script is re-run, and the
commit that re-runs it names the passage of the paper that justifies the
change.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2008_06134_gb300 import phantoms as ph  # noqa: E402

# (name, mode, light, render/build options): each a small scene of 16^3 blobs.
CASES = [
    ("none", oracle.NONE, None, {}),
    ("shadow", oracle.SHADOW, None, {}),
    ("shell", oracle.SHELL, None, {}),
    ("cone", oracle.CONE, None, {}),
    ("cone-depth-linear", oracle.CONE, None,
     {"quantity": oracle.OPTICAL_DEPTH, "slice_filter": oracle.SLICE_LINEAR}),
    ("shell-3", oracle.SHELL, None, {"shell_count": 3}),
    ("cone-point", oracle.CONE, (0.5, -1.2, 1.4), {}),
]


def scene():
    vol = ph.gaussian_blobs(16, seed=9, sigma=(1.5, 4.0))
    tf = ph.tf_random_pl(64, seed=9, alpha_max=0.3)
    cam = ph.orbit_camera(np.array([0.4, -0.7, -0.6]), True, 2.2)
    return vol, tf, cam


def main():
    vol, tf, cam = scene()
    W, H, n, R = 12, 9, 11, 13
    out = {"scene": "16^3 gaussian_blobs(seed 9, sigma 1.5-4), tf_random_pl(64, seed 9, "
                    "alpha_max 0.3), 11 slices of 13^2, light (0.3, -0.2, 0.9) unless a "
                    "point light, 12 x 9 perspective, step 0.5, ERT 0.95",
           "cases": {}}
    for name, mode, pos, opts in CASES:
        light = (oracle.light_setup((0.3, -0.2, 0.9), n, R) if pos is None
                 else oracle.point_light_setup(pos, n, R))
        q = opts.get("quantity", 0)
        B = None if mode == oracle.NONE else oracle.build_stack(vol, tf, 0, 255, light,
                                                                quantity=q)
        ro = oracle.render_opts(mode, 0.5, 0.95, (0.1, 0.2, 0.3, 0.0), ert_band=0.0, **opts)
        img, _, _, ns = oracle.render_image(vol, tf, 0, 255, light, B, cam, W, H, ro)
        case = {"image_rgba": img.reshape(-1).tolist(), "samples": ns.reshape(-1).tolist()}
        if B is not None:
            case["stack_every_7th"] = B.reshape(-1)[::7].tolist()
        out["cases"][name] = case
    with open(os.path.join(HERE, "oracle_small.json"), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()
