"""Oracle pins for volumetric shadows by ray forwarding: each sample's
emission is scaled by k_a + (1 - k_a) T_light, T_light the transmittance of
a shadow ray toward a directional light sampled at p + (i + 1/2) h L while
inside the volume box.

* T_light against brute force written here (numpy positions, scipy
  map_coordinates trilinear values, numpy.interp TF lookup, explicit
  product), at random points, for two light directions;
* the data-parallel form (shadow samples evaluated by their owner bricks,
  per-brick fragments, sort-last) equals the plain definition on the whole
  field (1e-12), regular and k-d partitions, cameras outside and inside;
* closed form: a constant field seen along x with the light along +z gives
  C = c (k_a + (1 - k_a)(1 - a_s)^n_s)(1 - (1 - a_p)^N) on the centre pixel,
  which a wrong light sign, a missing half step or the primary step in
  place of h would all change;
* k_a = 1 reduces to the unshadowed sort-last render bit for bit.
"""
import math

import numpy as np
import pytest
from scipy.ndimage import map_coordinates

from paper_2407_00179_b300 import inputs

DIMS = (30, 26, 34)


def _setup(seed=0, cut=0.05):
    f = inputs.blob_field(DIMS, inputs.blob_params(8, DIMS, seed)).numpy()
    return f, inputs.make_tf(1234, transparent_below=cut)


def _brute_T(field, tf, p, L, h, sigma, spacing):
    dims = np.array([field.shape[2], field.shape[1], field.shape[0]], np.float64)
    n = tf.shape[0]
    xs = np.arange(n) / (n - 1)
    T, cnt, i = 1.0, 0, 0
    while True:
        q = p + (i + 0.5) * h * L
        if np.any(q < 0.0) or np.any(q > dims - 1.0):
            break
        s = map_coordinates(field.astype(np.float64), [[q[2]], [q[1]], [q[0]]], order=1, mode="nearest")[0]
        a = np.interp(np.clip(s, 0.0, 1.0), xs, tf[:, 3].astype(np.float64))
        T *= math.exp(-sigma * a * h * spacing)
        cnt += 1
        i += 1
    return T, cnt


@pytest.mark.parametrize("direction", [(0.3, -0.5, 0.8), (-1.0, 0.2, 0.1)])
def test_light_transmittance_brute_force(orc, direction):
    f, tf = _setup(1)
    light = orc.Light(direction, step_voxels=0.75, ambient=0.2)
    L = np.asarray(direction, np.float64)
    L /= np.linalg.norm(L)
    rng = np.random.default_rng(3)
    pts = rng.uniform(0.0, 1.0, (40, 3)) * (np.array(DIMS) - 1)
    T, cnt, amb = orc.light_transmittance(DIMS, tf, pts, light, sigma_max=30.0, field=f)
    sp = 1.0 / (max(DIMS) - 1)
    for k, p in enumerate(pts):
        Tb, cb = _brute_T(f, tf, p, L, 0.75, 30.0, sp)
        assert cnt[k] == cb
        assert abs(T[k] - Tb) <= 1e-12
    assert T.min() < 0.7                       # the field actually shadows


PARTS = {
    "2x2x2": lambda d: inputs.regular_partition(d, (2, 2, 2)),
    "kd6": lambda d: inputs.kd_partition(d, 6, seed=2),
}


@pytest.mark.parametrize("pname", list(PARTS))
@pytest.mark.parametrize("inside", [False, True])
def test_partitioned_equals_plain(orc, pname, inside):
    f, tf = _setup(2)
    bricks = orc.make_bricks(f, PARTS[pname](DIMS), orc.F32)
    fr = orc.Frame(19, 15, step_voxels=0.5, sigma_max=20.0)
    light = orc.Light((0.4, 0.7, -0.6), step_voxels=1.0, ambient=0.3)
    for cam in inputs.random_cameras(DIMS, 2, seed=5 + len(pname), inside=inside):
        a = orc.render_shadow(DIMS, tf, cam, fr, light, field=f)
        b = orc.render_shadow(DIMS, tf, cam, fr, light, bricks=bricks)
        assert np.abs(a["rgba"] - b["rgba"]).max() <= 1e-12
        np.testing.assert_array_equal(a["nsamples"], b["nsamples"])
        np.testing.assert_array_equal(a["nshadow"], b["nshadow"])
        # shadows darken: the colour never exceeds the unshadowed one
        u = orc.render_bricks(DIMS, bricks, tf, cam, fr)
        assert np.all(b["rgba"][:, :3] <= u["rgba"][:, :3] + 1e-15)
        np.testing.assert_array_equal(b["rgba"][:, 3], u["rgba"][:, 3])
        if not inside:
            assert (u["rgba"][:, :3] - b["rgba"][:, :3]).max() > 1e-3


def test_constant_field_closed_form(orc):
    dims = (40, 9, 21)
    s0 = 0.5
    f = np.full((dims[2], dims[1], dims[0]), s0, np.float32)
    n = 257
    tab = np.zeros((n, 4), np.float32)
    tab[:, 0], tab[:, 1], tab[:, 2], tab[:, 3] = 0.75, 0.5, 0.25, 0.5
    sp = 1.0 / (max(dims) - 1)
    zc = 6.7
    cam = inputs.Camera((-3.0, 4.0 * sp, zc * sp), (0.5, 4.0 * sp, zc * sp), (0.0, 0.0, 1.0), 2.0)
    fr = orc.Frame(5, 5, step_voxels=0.5, sigma_max=16.0)
    ka, h = 0.25, 1.0
    light = orc.Light((0.0, 0.0, 1.0), step_voxels=h, ambient=ka)
    bricks = orc.make_bricks(f, inputs.regular_partition(dims, (4, 1, 2)), orc.F32)
    for src in (dict(field=f), dict(bricks=bricks)):
        r = orc.render_shadow(dims, tab, cam, fr, light, **src)
        k = 12                                   # centre pixel of 5 x 5
        N = int(r["nsamples"][k])
        assert N == 78                           # 39 node units at step 0.5
        a_p = 1.0 - math.exp(-16.0 * 0.5 * 0.5 * sp)
        a_s = 1.0 - math.exp(-16.0 * 0.5 * h * sp)
        n_s = 13                                 # 6.7 + i + 1/2 <= 20 for i = 0..12
        assert r["nshadow"][k] == N * n_s
        A = 1.0 - (1.0 - a_p) ** N
        w = ka + (1.0 - ka) * (1.0 - a_s) ** n_s
        np.testing.assert_allclose(r["rgba"][k], [0.75 * w * A, 0.5 * w * A, 0.25 * w * A, A], rtol=0, atol=1e-13)


def test_full_ambient_is_unshadowed(orc):
    f, tf = _setup(3)
    bricks = orc.make_bricks(f, PARTS["kd6"](DIMS), orc.F32)
    fr = orc.Frame(17, 13, step_voxels=0.5, sigma_max=20.0, ert=0.9)
    cam = inputs.camera_from_direction(DIMS, (1.0, 0.7, 0.5))
    a = orc.render_shadow(DIMS, tf, cam, fr, orc.Light((0.0, 1.0, 0.0), ambient=1.0), bricks=bricks)
    b = orc.render_bricks(DIMS, bricks, tf, cam, fr)
    np.testing.assert_array_equal(a["rgba"], b["rgba"])
    np.testing.assert_array_equal(a["depth"], b["depth"])
    np.testing.assert_array_equal(a["nsamples"], b["nsamples"])
