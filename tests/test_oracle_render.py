"""Oracle pins for the forward render.

* camera convention: geometric properties of the rays, and the rays of
  the OpenGL look-at / perspective unprojection;
* closed form 1 (constant slab): A = 1 - exp(-sigma d), C = c A;
* closed form 2 (linear extinction): the midpoint samples integrate a linear
  sigma exactly, on axis-aligned and oblique rays;
* convergence to the continuous emission-absorption integral at second order;
* brute force on tiny volumes: samples enumerated directly, trilinear from
  scipy.ndimage.map_coordinates, TF from numpy.interp, and compositing as the
  explicit product sum C = sum_i alpha_i c_i prod_{j<i} (1 - alpha_j).
"""
import math

import numpy as np
import pytest
from scipy.ndimage import map_coordinates

from paper_2407_00179_b300 import inputs


def _frame(orc, W, H, **kw):
    return orc.Frame(W, H, **kw)


def _const_tf(rgba, n=256):
    return np.tile(np.asarray(rgba, np.float32), (n, 1))


# --------------------------------------------------------------------------
# camera convention
# --------------------------------------------------------------------------

def test_camera_rays_geometry(orc):
    cam = inputs.Camera((3.0, -1.0, 2.0), (0.2, 0.4, 0.1), (0.0, 0.0, 1.0), 40.0)
    W, H = 9, 7
    f = np.array(cam.center) - np.array(cam.eye)
    f /= np.linalg.norm(f)
    r = np.cross(f, cam.up)
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    o, d = orc.camera_ray(cam, W, H, 4, 3)           # centre pixel (odd sizes)
    np.testing.assert_allclose(o, cam.eye, atol=0)
    np.testing.assert_allclose(d, f, atol=1e-15)
    for px, py in [(0, 0), (8, 6), (2, 5)]:
        _, d = orc.camera_ray(cam, W, H, px, py)
        assert abs(np.linalg.norm(d) - 1) < 1e-15
        # row 0 is the bottom, column 0 the left
        assert np.sign(d @ u) == np.sign(py - 3)
        assert np.sign(d @ r) == np.sign(px - 4)
    # the top edge of the image is at fovy/2 above the axis: the top row's
    # pixel centre is (H - 1/2)/H of the way there in tangent space
    _, d = orc.camera_ray(cam, W, H, 4, H - 1)
    ang = math.atan2(d @ u, d @ f)
    assert abs(math.tan(ang) - ((H - 0.5) / H * 2 - 1) * math.tan(math.radians(20))) < 1e-14
    # horizontal field of view scales with the aspect ratio W / H
    _, d = orc.camera_ray(cam, W, H, W - 1, 3)
    assert abs(math.atan2(d @ r, d @ f) - math.atan(((W - 0.5) / W * 2 - 1) * W / H * math.tan(math.radians(20)))) < 1e-14


def _gl_look_at(eye, center, up):
    """The viewing matrix of the fixed-function OpenGL look-at (world to eye
    coordinates, the eye looking down -z), as its reference page defines it."""
    f = np.asarray(center, np.float64) - np.asarray(eye, np.float64)
    f /= np.linalg.norm(f)
    s = np.cross(f, np.asarray(up, np.float64))
    s /= np.linalg.norm(s)
    u = np.cross(s, f)
    m = np.eye(4)
    m[0, :3], m[1, :3], m[2, :3] = s, u, -f
    t = np.eye(4)
    t[:3, 3] = -np.asarray(eye, np.float64)
    return m @ t


def _gl_perspective(fovy_deg, aspect, near, far):
    """The fixed-function OpenGL perspective projection (eye to clip
    coordinates), as its reference page defines it."""
    f = 1.0 / math.tan(math.radians(fovy_deg) / 2.0)
    p = np.zeros((4, 4))
    p[0, 0] = f / aspect
    p[1, 1] = f
    p[2, 2] = (far + near) / (near - far)
    p[2, 3] = 2.0 * far * near / (near - far)
    p[3, 2] = -1.0
    return p


def _gl_unproject(win, inv_pv, W, H):
    """Window coordinates (x, y from the lower-left corner, depth in [0, 1])
    to world coordinates through the inverse of projection x view."""
    ndc = np.array([2.0 * win[0] / W - 1.0, 2.0 * win[1] / H - 1.0, 2.0 * win[2] - 1.0, 1.0])
    w = inv_pv @ ndc
    return w[:3] / w[3]


@pytest.mark.parametrize("W,H", [(9, 7), (64, 36), (5, 11)])
def test_camera_rays_match_the_gl_unprojection(orc, W, H):
    """The camera convention pinned to a textbook one: the OpenGL look-at
    and perspective matrices (vertical field of view, aspect W / H), whose
    window origin is the lower-left corner.  A pixel centre unprojected at
    the near and the far plane gives a segment; its direction, and the eye
    as its origin, equal the oracle's ray for that pixel.  A transposed
    basis, a flipped row order, a half-angle slip or the aspect on the wrong
    axis fails here."""
    rng = inputs.rng(11, inputs.STREAM_SELECT)
    for trial in range(6):
        eye = rng.normal(size=3) * 3.0
        center = rng.normal(size=3) * 0.5
        up = rng.normal(size=3)
        fovy = float(rng.uniform(15.0, 80.0))
        cam = inputs.Camera(tuple(eye), tuple(center), tuple(up), fovy)
        inv_pv = np.linalg.inv(_gl_perspective(fovy, W / H, 0.5, 50.0) @ _gl_look_at(eye, center, up))
        for px, py in [(0, 0), (W - 1, H - 1), (W // 2, 0), (1, H - 2), (W - 1, 0)]:
            a = _gl_unproject((px + 0.5, py + 0.5, 0.0), inv_pv, W, H)
            b = _gl_unproject((px + 0.5, py + 0.5, 1.0), inv_pv, W, H)
            ref = (b - a) / np.linalg.norm(b - a)
            o, d = orc.camera_ray(cam, W, H, px, py)
            np.testing.assert_allclose(d, ref, atol=1e-9)
            # the segment lies on the ray from the eye
            np.testing.assert_allclose(np.cross(a - np.asarray(o), d), 0.0, atol=1e-8)


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------

DIMS = (9, 5, 5)            # spacing 1/8, x spans [0, 1], y and z span [0, 0.5]


def _axis_camera():
    # looks down -x through the middle of the y/z extent; one pixel, on axis
    return inputs.Camera((2.0, 0.25, 0.25), (0.5, 0.25, 0.25), (0.0, 0.0, 1.0), 40.0)


@pytest.mark.parametrize("s0", [0.0, 0.3, 0.77, 1.0])
@pytest.mark.parametrize("sigma_max", [0.5, 8.0, 40.0])
def test_constant_slab(orc, s0, sigma_max):
    tf = inputs.make_tf(seed=5)
    f = np.full(DIMS[::-1], s0, np.float32)
    fr = _frame(orc, 1, 1, step_voxels=0.4, sigma_max=sigma_max)       # dt = 0.05, d = 1 = 20 dt
    out = orc.render_full(f, tf, _axis_camera(), fr)
    assert out["nsamples"][0] == 20
    v = [np.interp(np.float32(s0), np.arange(256) / 255.0, tf[:, c].astype(np.float64)) for c in range(4)]
    sig = sigma_max * v[3]
    A = 1.0 - math.exp(-sig * 1.0)                                   # Beer-Lambert over d = 1
    np.testing.assert_allclose(out["rgba"][0, 3], A, rtol=0, atol=1e-13)
    np.testing.assert_allclose(out["rgba"][0, :3], np.array(v[:3]) * A, rtol=0, atol=1e-13)


def _linear_field(a, b):
    x = np.arange(DIMS[0]) / (DIMS[0] - 1)
    f = a + b * x
    return np.broadcast_to(f[None, None, :], DIMS[::-1]).astype(np.float32).copy()


def _ramp_tf(c0):
    # 257 entries: alpha_i = i / 256 is exact in float32, so alpha(s) = s
    tf = np.zeros((257, 4), np.float32)
    tf[:, :3] = c0
    tf[:, 3] = np.arange(257) / 256.0
    return tf


def test_linear_sigma_axis(orc):
    a, b, sm = 0.125, 0.75, 6.0
    c0 = np.array([0.2, 0.5, 0.9], np.float32)
    f = _linear_field(a, b)
    fr = _frame(orc, 1, 1, step_voxels=0.4, sigma_max=sm)
    out = orc.render_full(f, _ramp_tf(c0), _axis_camera(), fr)
    # integral of sigma_max * (a + b x) over x in [0, 1]
    tau = sm * (a + b / 2)
    A = 1 - math.exp(-tau)
    np.testing.assert_allclose(out["rgba"][0, 3], A, atol=1e-13)
    np.testing.assert_allclose(out["rgba"][0, :3], c0.astype(np.float64) * A, atol=1e-13)


def test_linear_sigma_oblique(orc):
    """Oblique rays through a field linear in all three coordinates: the sum
    over midpoint samples equals N dt sigma(centre of the sampled interval)."""
    dims = (9, 8, 7)
    sp = 1 / 8                       # dyadic, so the field is exact in float32
    g = np.array([0.3125, -0.1875, 0.25])
    zz, yy, xx = np.meshgrid(np.arange(dims[2]), np.arange(dims[1]), np.arange(dims[0]), indexing="ij")
    pos = np.stack([xx, yy, zz], -1) * sp
    f = (0.375 + pos @ g).astype(np.float32)
    assert f.min() >= 0 and f.max() <= 1
    c0 = np.array([0.7, 0.1, 0.3], np.float32)
    cam = inputs.camera_from_direction(dims, (0.8, 0.45, -0.3))
    W, H = 11, 9
    fr = _frame(orc, W, H, step_voxels=0.7, sigma_max=5.0)
    out = orc.render_full(f, _ramp_tf(c0), cam, fr)
    lo = np.zeros(3)
    hi = (np.array(dims) - 1) * sp
    checked = 0
    for p in range(W * H):
        o, d = orc.camera_ray(cam, W, H, p % W, p // W)
        with np.errstate(divide="ignore"):
            t0 = (lo - o) / d
            t1 = (hi - o) / d
        te = max(0.0, np.minimum(t0, t1).max())
        tx = np.maximum(t0, t1).min()
        if te >= tx:
            assert out["nsamples"][p] == 0 and np.all(out["rgba"][p] == 0)
            continue
        dt = 0.7 * sp
        n = int(out["nsamples"][p])
        # the sample count is the number of midpoints before the exit
        assert te + (n - 0.5) * dt < tx <= te + (n + 0.5) * dt
        mid = te + 0.5 * n * dt
        s_mid = 0.375 + (o + mid * d) @ g
        A = 1 - math.exp(-5.0 * s_mid * n * dt)
        assert abs(out["rgba"][p, 3] - A) < 1e-12
        checked += 1
    assert checked > W * H // 3


def test_convergence_second_order(orc):
    """alpha constant, colour linear along the ray: the discrete sum tends to
    C = c0 (1 - e^{-sd}) + g (1 - e^{-sd} (1 + s d)) / s at second order."""
    a0, sm = 0.5, 8.0
    f = _linear_field(0.0, 1.0)           # s = x in world units
    tf = np.zeros((257, 4), np.float32)
    tf[:, 0] = np.arange(257) / 256.0     # red = s, exact in float32
    tf[:, 3] = a0
    sig, d = sm * a0, 1.0
    # along the ray x = 1 - tau, so c(tau) = 1 - tau
    exact = 1.0 * (1 - math.exp(-sig * d)) - (1 - math.exp(-sig * d) * (1 + sig * d)) / sig
    errs = []
    for step in (0.4, 0.2, 0.1, 0.05):
        out = orc.render_full(f, tf, _axis_camera(), _frame(orc, 1, 1, step_voxels=step, sigma_max=sm))
        errs.append(abs(out["rgba"][0, 0] - exact))
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(3.6 < r < 4.4 for r in ratios), (errs, ratios)


# --------------------------------------------------------------------------
# brute force
# --------------------------------------------------------------------------

def _brute_pixel(orc, field64, tf, cam, W, H, px, py, step, sm, sp):
    dims = field64.shape[::-1]
    o, d = orc.camera_ray(cam, W, H, px, py)
    lo = np.zeros(3)
    hi = (np.array(dims) - 1) * sp
    with np.errstate(divide="ignore", invalid="ignore"):
        t0 = (lo - o) / d
        t1 = (hi - o) / d
    te = max(0.0, np.nanmax(np.minimum(t0, t1)))
    tx = np.nanmin(np.maximum(t0, t1))
    if te >= tx:
        return np.zeros(4), 0
    dt = step * sp
    ts = []
    j = 0
    while te + (j + 0.5) * dt < tx:
        ts.append(te + (j + 0.5) * dt)
        j += 1
    if not ts:
        return np.zeros(4), 0
    q = (o[None, :] + np.array(ts)[:, None] * d[None, :]) / sp
    q = np.clip(q, 0, np.array(dims) - 1)
    s = map_coordinates(field64, [q[:, 2], q[:, 1], q[:, 0]], order=1, mode="nearest")
    u = np.clip(s, 0, 1) * (tf.shape[0] - 1)
    knots = np.arange(tf.shape[0])
    rgba = np.stack([np.interp(u, knots, tf[:, c].astype(np.float64)) for c in range(4)], -1)
    alpha = 1 - np.exp(-sm * rgba[:, 3] * dt)
    C = np.zeros(3)
    for i in range(len(ts)):
        trans = 1.0
        for k in range(i):
            trans *= 1 - alpha[k]
        C += alpha[i] * rgba[i, :3] * trans
    A = 1 - np.prod(1 - alpha)
    return np.concatenate([C, [A]]), len(ts)


@pytest.mark.parametrize("case", [0, 1, 2])
def test_brute_force_tiny(orc, case):
    g = np.random.default_rng(100 + case)
    dims = [(5, 4, 6), (6, 6, 6), (4, 7, 5)][case]
    field = g.uniform(0, 1, dims[::-1]).astype(np.float32)
    tf = inputs.make_tf(seed=7 + case)
    cams = [inputs.camera_from_direction(dims, (1, 0.7, 0.5)),
            inputs.random_cameras(dims, 1, seed=case, inside=True)[0],
            inputs.random_cameras(dims, 1, seed=case)[0]]
    W, H = 7, 5
    sp = 1.0 / (max(dims) - 1)
    step, sm = 0.37, 9.0
    fr = _frame(orc, W, H, step_voxels=step, sigma_max=sm)
    part = inputs.regular_partition(dims, (2, 1, 2))
    bricks = orc.make_bricks(field, part, orc.F32)
    for cam in cams:
        full = orc.render_full(field, tf, cam, fr)
        br = orc.render_bricks(dims, bricks, tf, cam, fr)
        for p in range(W * H):
            ref, n = _brute_pixel(orc, field.astype(np.float64), tf, cam, W, H, p % W, p // W, step, sm, sp)
            assert full["nsamples"][p] == n
            np.testing.assert_allclose(full["rgba"][p], ref, atol=1e-13, rtol=0)
            np.testing.assert_allclose(br["rgba"][p], ref, atol=1e-13, rtol=0)
            assert br["nsamples"][p] == n
