"""Oracle pins for the gradient (the differentiable form of the path).

The oracle's reverse-mode gradient (a reverse sweep over a per-sample tape)
is checked against FP64 central finite differences of the oracle's own
forward render, for transfer-function entries and for voxels, with early
termination off and on.  A planted sign error on the CPU must fail."""
import numpy as np
import pytest

from paper_2407_00179_b300 import inputs


def _problem(seed=0, dims=(10, 9, 8), ert=0.0, splits=(2, 2, 1)):
    f = inputs.blob_field(dims, inputs.blob_params(4, dims, seed, sigma_range=(0.2, 0.4))).numpy()
    tf = inputs.make_tf(seed=77 + seed)
    part = inputs.regular_partition(dims, splits)
    cam = inputs.camera_from_direction(dims, (1, 0.6, 0.45))
    W, H = 9, 7
    g = np.random.default_rng(seed).normal(size=(W * H, 4))
    return dims, f, tf, part, cam, W, H, g, ert


def _loss(orc, dims, f, tf, part, cam, fr, g):
    br = orc.render_bricks(dims, orc.make_bricks(f, part, orc.F32), tf, cam, fr)
    return float(np.sum(br["rgba"] * g))


@pytest.mark.parametrize("ert", [0.0, 0.6])
def test_tf_gradient_matches_fd(orc, ert):
    dims, f, tf, part, cam, W, H, g, _ = _problem(0, ert=ert)
    fr = orc.Frame(W, H, sigma_max=20.0, ert=ert)
    bricks = orc.make_bricks(f, part, orc.F32)
    dtf, _ = orc.grad_bricks(dims, bricks, tf, cam, fr, g, want_volume=False)
    rng = np.random.default_rng(1)
    nz = np.argwhere(np.abs(dtf) > 1e-3 * np.abs(dtf).max())
    picks = nz[rng.choice(len(nz), size=min(40, len(nz)), replace=False)]
    eps = 1e-6
    for i, c in picks:
        tp = tf.astype(np.float64).copy()
        # perturb in float64 space; the oracle reads a float32 table, so use
        # a perturbation that is exact in float32
        e = np.float32(eps)
        t1 = tf.copy(); t1[i, c] += e
        t0 = tf.copy(); t0[i, c] -= e
        h = (np.float64(t1[i, c]) - np.float64(t0[i, c]))
        fd = (_loss(orc, dims, f, t1, part, cam, fr, g) - _loss(orc, dims, f, t0, part, cam, fr, g)) / h
        assert abs(fd - dtf[i, c]) <= 1e-5 * abs(dtf).max() + 1e-4 * abs(fd), (i, c, fd, dtf[i, c])


@pytest.mark.parametrize("ert", [0.0, 0.6])
def test_voxel_gradient_matches_fd(orc, ert):
    dims, f, tf, part, cam, W, H, g, _ = _problem(1, ert=ert)
    fr = orc.Frame(W, H, sigma_max=20.0, ert=ert)
    bricks = orc.make_bricks(f, part, orc.F32)
    _, dvol = orc.grad_bricks(dims, bricks, tf, cam, fr, g)
    rng = np.random.default_rng(2)
    nz = np.argwhere(np.abs(dvol) > 1e-3 * np.abs(dvol).max())
    picks = nz[rng.choice(len(nz), size=min(40, len(nz)), replace=False)]
    eps = np.float32(1e-4)
    errs = []
    for z, y, x in picks:
        f1 = f.copy(); f1[z, y, x] += eps
        f0 = f.copy(); f0[z, y, x] -= eps
        h = np.float64(f1[z, y, x]) - np.float64(f0[z, y, x])
        fd = (_loss(orc, dims, f1, tf, part, cam, fr, g) - _loss(orc, dims, f0, tf, part, cam, fr, g)) / h
        errs.append(abs(fd - dvol[z, y, x]) / (abs(dvol).max()))
    errs = np.array(errs)
    # a TF knot crossed within +-eps makes central differences inexact for a
    # few voxels; the rest agree to rounding
    assert np.median(errs) < 1e-8
    assert np.sum(errs > 1e-6) <= 2
    assert errs.max() < 2e-3


def test_ghost_gradients_reach_owner(orc):
    """Voxels in a ghost layer get the gradient of both bricks' samples: the
    partitioned gradient equals the gradient of the unpartitioned problem
    (one brick), since the forward images are equal."""
    dims, f, tf, part, cam, W, H, g, _ = _problem(2)
    fr = orc.Frame(W, H, sigma_max=20.0)
    d8 = orc.grad_bricks(dims, orc.make_bricks(f, part, orc.F32), tf, cam, fr, g)
    one = inputs.regular_partition(dims, (1, 1, 1))
    d1 = orc.grad_bricks(dims, orc.make_bricks(f, one, orc.F32), tf, cam, fr, g)
    assert np.abs(d8[0] - d1[0]).max() <= 1e-10 * np.abs(d1[0]).max()
    assert np.abs(d8[1] - d1[1]).max() <= 1e-10 * np.abs(d1[1]).max()


def test_planted_sign_error_fails_fd(orc):
    """Planted mistake on the CPU: flipping the sign of the opacity gradient
    (as a wrong adjoint would) is caught by the finite differences."""
    dims, f, tf, part, cam, W, H, g, _ = _problem(0)
    fr = orc.Frame(W, H, sigma_max=20.0)
    bricks = orc.make_bricks(f, part, orc.F32)
    dtf, _ = orc.grad_bricks(dims, bricks, tf, cam, fr, g, want_volume=False)
    i = int(np.argmax(np.abs(dtf[:, 3])))
    e = np.float32(1e-6)
    t1 = tf.copy(); t1[i, 3] += e
    t0 = tf.copy(); t0[i, 3] -= e
    fd = (_loss(orc, dims, f, t1, part, cam, fr, g) - _loss(orc, dims, f, t0, part, cam, fr, g)) / (
        np.float64(t1[i, 3]) - np.float64(t0[i, 3]))
    assert abs(fd - dtf[i, 3]) < 1e-4 * abs(fd)
    assert abs(fd - (-dtf[i, 3])) > 0.5 * abs(fd)


def _knot_problem(orc, value, tab, toward=None):
    """Field of `value` and its float32 neighbour toward `toward` in a
    checkerboard (constant if toward is None)."""
    dims = (6, 5, 4)
    f = np.full((dims[2], dims[1], dims[0]), value, np.float32)
    if toward is not None:
        z, y, x = np.indices(f.shape)
        f[(x + y + z) % 2 == 1] = np.nextafter(np.float32(value), np.float32(toward))
    part = inputs.regular_partition(dims, (2, 1, 1))
    cam = inputs.camera_from_direction(dims, (1, 0.6, 0.45))
    W, H = 9, 7
    g = np.random.default_rng(5).normal(size=(W * H, 4))
    fr = orc.Frame(W, H, sigma_max=20.0)
    return orc.grad_bricks(dims, orc.make_bricks(f, part, orc.F32), tab, cam, fr, g, knot_eps=orc.KNOT_EPS)


def test_knot_ambiguity_covers_the_one_sided_jump(orc):
    """At a TF knot where the slope changes, the field gradient jumps between
    the two one-sided derivatives.  A constant field one float32 step above
    and one below the knot (checkerboards of two neighbouring float32
    values) gives the two sides; their difference must be covered by the
    reported knot ambiguity (triangle inequality over the samples), which is
    exactly zero for a field away from every knot, for a TF whose slope does
    not change at the knot, and for samples whose corners are all equal.
    Tables are dyadic, so equal slopes are equal in floating point."""
    n = 257
    u = np.arange(n) / 256.0
    kinked = np.stack([u, np.full(n, 0.3), 1.0 - u, 0.25 + 0.5 * np.abs(u - 0.5)], 1).astype(np.float32)
    linear = np.stack([u, np.full(n, 0.3), 1.0 - u, 0.25 + 0.5 * u], 1).astype(np.float32)
    half = np.float32(0.5)                    # knot 128
    above, below = np.nextafter(half, np.float32(1)), np.nextafter(half, np.float32(0))
    _, dv_hi, amb_hi = _knot_problem(orc, above, kinked, toward=1.0)
    _, dv_lo, amb_lo = _knot_problem(orc, below, kinked, toward=0.0)
    m = np.abs(dv_hi).max()
    jump = np.abs(dv_hi - dv_lo)
    assert jump.max() > 1e-2 * m                      # the kink is real
    assert np.all(jump <= amb_hi * (1 + 1e-6) + 1e-9 * m)
    assert np.all(jump <= amb_lo * (1 + 1e-6) + 1e-9 * m)
    assert amb_hi.max() <= 4 * jump.max()             # and not a blanket bound
    # away from every knot: mid-segment value
    _, _, amb_mid = _knot_problem(orc, np.float32(0.5 + 0.5 / 256), kinked, toward=1.0)
    assert amb_mid.max() == 0.0
    # no slope change at the knot: nothing is ambiguous
    _, dv_lin, amb_lin = _knot_problem(orc, above, linear, toward=1.0)
    assert np.abs(dv_lin).max() > 0 and amb_lin.max() == 0.0
    # equal corners: s is exact, so it stays on its side of the knot
    _, dv_flat, amb_flat = _knot_problem(orc, above, kinked)
    assert np.abs(dv_flat).max() > 0 and amb_flat.max() == 0.0


def test_tf_coordinate_ambiguity_closed_form(orc):
    """With a two-entry table every sample splits its value adjoint between
    entries 0 and 1 (u in [0, 1], du = 2^-22); where every adjoint of a
    channel has one sign (colour channels under a non-negative image
    gradient: T alpha g >= 0) the ambiguity of each entry is exactly
    2^-22 |dtf[0] + dtf[1]| of that channel.  It is zero for an untouched
    entry and never negative."""
    dims, f, tf, part, cam, W, H, g, _ = _problem(2)
    fr = orc.Frame(W, H, sigma_max=20.0)
    bricks = orc.make_bricks(f, part, orc.F32)
    g = np.abs(g)
    g[:, 3] = 0.0
    tf2 = inputs.make_tf(5, n=2)
    dtf, _, amb = orc.grad_bricks(dims, bricks, tf2, cam, fr, g, want_volume=False, tf_amb=True)
    for c in range(3):
        want = 2.0 ** -22 * abs(dtf[0, c] + dtf[1, c])
        assert want > 0
        np.testing.assert_allclose(amb[:, c], [want, want], rtol=1e-12)
    # a 256-entry table: non-negative, zero where no sample reads
    dtf, _, amb = orc.grad_bricks(dims, bricks, tf, cam, fr, np.abs(g), want_volume=False, tf_amb=True)
    assert np.all(amb >= 0.0)
    assert np.all(amb[np.all(dtf == 0.0, axis=1)] == 0.0)
    assert amb.max() > 0
