"""Write the stored expected values of tests/golden/ from the FP64 oracle.

The paper prints no numeric example for its rendering path (it has no
equations, §8), so the stored values are the oracle's own output for a small
seeded scene of the sort-last method (§2.1 one fragment per rank and pixel,
§5.1.1 key-ordered front-to-back compositing), written once by this script
and then checked against the oracle (a regression pin) and the CUDA path.
Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2407_00179_b300 import inputs  # noqa: E402

DIMS = (24, 20, 28)
WIDTH, HEIGHT = 16, 12


def scene():
    """Field, partition, TF, float32 camera, frame and spacing of the golden scene."""
    f = inputs.blob_field(DIMS, inputs.blob_params(6, DIMS, 7)).numpy()
    part = inputs.regular_partition(DIMS, (2, 1, 2))
    tf = inputs.make_tf(1234)
    c = inputs.camera_from_direction(DIMS, (1.0, 0.7, 0.5))
    f32 = lambda v: tuple(float(x) for x in np.asarray(v, np.float32))
    cam = inputs.Camera(f32(c.eye), f32(c.center), f32(c.up), float(np.float32(c.fovy_deg)))
    spacing = float(np.float32(1.0 / (max(DIMS) - 1)))
    fr = oracle.Frame(WIDTH, HEIGHT, step_voxels=0.5, sigma_max=20.0)
    return f, part, tf, cam, fr, spacing


def render():
    f, part, tf, cam, fr, spacing = scene()
    bricks = oracle.make_bricks(f, part, oracle.F32)
    return oracle.render_bricks(DIMS, bricks, tf, cam, fr, spacing=spacing)


def main():
    r = render()
    path = os.path.join(HERE, "small_frame.txt")
    with open(path, "w") as out:
        out.write("# Sort-last frame of a seeded 24x20x28 blob field, 2x1x2 bricks, 16x12 pixels,\n")
        out.write("# step 0.5 voxel, sigma_max 20, TF seed 1234, camera from direction (1, 0.7, 0.5).\n")
        out.write("# Written by tests/golden/make_golden.py from the FP64 oracle (oracle/ only):\n")
        out.write("# one fragment per rank and pixel (paper §2.1), composited front to back in key\n")
        out.write("# order (§5.1.1).  Columns: pixel, flags, R G B A (premultiplied), depth,\n")
        out.write("# brick order (0xFF = none).\n")
        for k in range(WIDTH * HEIGHT):
            rgba = " ".join("%.17g" % v for v in r["rgba"][k])
            order = " ".join(str(int(v)) for v in r["order"][k])
            out.write("%d %d %s %.17g %s\n" % (k, int(r["flags"][k]), rgba, r["depth"][k], order))
    print("wrote", path)


if __name__ == "__main__":
    main()
