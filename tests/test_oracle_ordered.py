"""Oracle pins for the visibility-ordered march with global early
termination (bricks marched in each ray's front-to-back order, carrying the
transmittance, stopping once the accumulated opacity passes the threshold).

* without termination it equals the sort-last composite (over is
  associative: 1e-12), samples and depth identical;
* with termination the partitioned form equals the unpartitioned plain
  definition exactly (regular and k-d partitions, cameras outside and
  inside);
* closed form: a constant slab stops after the first n with
  1 - (1 - alpha)^n > threshold, with C = c (1 - (1 - alpha)^n);
* it evaluates no more samples than per-fragment termination, and on an
  opaque scene fewer, with a different image (the planted mix-up of the two
  rules is caught).
"""
import math

import numpy as np
import pytest

from paper_2407_00179_b300 import inputs

PARTS = {
    "2x2x2": lambda d: inputs.regular_partition(d, (2, 2, 2)),
    "3x2x4": lambda d: inputs.regular_partition(d, (3, 2, 4)),
    "kd9": lambda d: inputs.kd_partition(d, 9, seed=5),
}


def _setup(dims=(24, 20, 28), seed=0):
    f = inputs.blob_field(dims, inputs.blob_params(8, dims, seed)).numpy()
    return f, inputs.make_tf(1234)


def test_without_termination_equals_sort_last(orc):
    dims = (24, 20, 28)
    f, tf = _setup(dims)
    bricks = orc.make_bricks(f, PARTS["kd9"](dims), orc.F32)
    fr = orc.Frame(23, 19, step_voxels=0.5, sigma_max=8.0, ert=0.0)
    for cam in inputs.random_cameras(dims, 2, seed=3):
        a = orc.render_ordered(dims, tf, cam, fr, bricks=bricks)
        b = orc.render_bricks(dims, bricks, tf, cam, fr)
        assert np.abs(a["rgba"] - b["rgba"]).max() <= 1e-12
        np.testing.assert_array_equal(a["nsamples"], b["nsamples"])
        np.testing.assert_array_equal(a["depth"], b["depth"])
        assert b["rgba"][:, 3].max() > 0.05


@pytest.mark.parametrize("pname", list(PARTS))
@pytest.mark.parametrize("inside", [False, True])
def test_partitioned_equals_unpartitioned(orc, pname, inside):
    dims = (24, 20, 28)
    f, tf = _setup(dims, 2)
    bricks = orc.make_bricks(f, PARTS[pname](dims), orc.F32)
    fr = orc.Frame(23, 19, step_voxels=0.5, sigma_max=60.0, ert=0.95)
    stopped = 0
    for cam in inputs.random_cameras(dims, 2, seed=11 + list(PARTS).index(pname), inside=inside):
        a = orc.render_ordered(dims, tf, cam, fr, field=f)
        b = orc.render_ordered(dims, tf, cam, fr, bricks=bricks)
        np.testing.assert_array_equal(a["rgba"], b["rgba"])
        np.testing.assert_array_equal(a["nsamples"], b["nsamples"])
        np.testing.assert_array_equal(a["depth"], b["depth"])
        full = orc.render_full(f, tf, cam, fr)
        stopped += int((a["nsamples"] < full["nsamples"]).sum())
    assert stopped > 20                       # termination actually happens


def test_constant_slab_closed_form(orc):
    dims = (40, 9, 9)
    s0 = 0.5
    f = np.full((dims[2], dims[1], dims[0]), s0, np.float32)
    n = 257
    tab = np.zeros((n, 4), np.float32)
    tab[:, 0], tab[:, 1], tab[:, 2], tab[:, 3] = 0.75, 0.5, 0.25, 0.5     # constant, dyadic
    bricks = orc.make_bricks(f, inputs.regular_partition(dims, (4, 1, 1)), orc.F32)
    thr = 0.9
    fr = orc.Frame(5, 5, step_voxels=0.5, sigma_max=16.0, ert=thr)
    cam = inputs.Camera((-3.0, 4.0 / 39.0, 4.0 / 39.0), (0.5, 4.0 / 39.0, 4.0 / 39.0), (0.0, 0.0, 1.0), 2.0)
    r = orc.render_ordered(dims, tab, cam, fr, bricks=bricks)
    k = 12                                    # the centre pixel of 5 x 5
    sp = 1.0 / (max(dims) - 1)
    alpha = 1.0 - math.exp(-16.0 * 0.5 * 0.5 * sp)
    nstar = next(m for m in range(1, 1000) if 1.0 - (1.0 - alpha) ** m > thr)
    A = 1.0 - (1.0 - alpha) ** nstar
    assert r["nsamples"][k] == nstar
    np.testing.assert_allclose(r["rgba"][k], [0.75 * A, 0.5 * A, 0.25 * A, A], rtol=0, atol=1e-13)
    # it crossed brick faces while carrying the transmittance (n* spans bricks)
    assert nstar * 0.5 > 10


def test_fewer_samples_than_per_fragment_termination(orc):
    dims = (32, 28, 30)
    f, tf = _setup(dims, 4)
    bricks = orc.make_bricks(f, PARTS["2x2x2"](dims), orc.F32)
    fr = orc.Frame(31, 27, step_voxels=0.5, sigma_max=80.0, ert=0.9)
    cam = inputs.camera_from_direction(dims, (1, 0.7, 0.5))
    a = orc.render_ordered(dims, tf, cam, fr, bricks=bricks)
    b = orc.render_bricks(dims, bricks, tf, cam, fr)
    assert np.all(a["nsamples"] <= b["nsamples"])
    assert a["nsamples"].sum() < 0.9 * b["nsamples"].sum()
    # the two termination rules give different images on an opaque scene
    assert np.abs(a["rgba"] - b["rgba"]).max() > 1e-6
