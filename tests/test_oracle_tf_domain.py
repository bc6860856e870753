"""Oracle pins for the transfer-function domain [vmin, vmax] and its clamp.

The lookup maps a value s to the table through the domain [vmin, vmax]:
entries sit at s_i = vmin + i (vmax - vmin) / (n - 1), values between two
entries interpolate linearly, values outside the domain take the end entry,
and the derivative with respect to s is zero on the clamped sides.

* brute force on tiny volumes with a non-unit domain and a field that
  crosses both ends: samples enumerated directly, trilinear from
  scipy.ndimage.map_coordinates, and the table looked up with numpy.interp
  on s itself at the entries' s positions (numpy.interp holds the end
  values outside the knots, which is the clamp);
* FP64 central differences of the oracle's own loss for the field gradient
  at voxels whose samples all lie below vmin, all above vmax, or inside,
  and for the TF entries at both ends of the table;
* planted mistakes, compiled into a copy of the oracle source on the CPU: a
  domain mapped as (s - vmin) (n - 1) / vmax fails the brute force, and a
  derivative not zeroed on the clamped side fails the central differences.
"""
import os

import numpy as np
import pytest
from scipy.ndimage import map_coordinates

from paper_2407_00179_b300 import inputs

DOMAINS = [(0.2, 0.8), (-0.25, 1.6)]


def _field(dims, seed, lo, hi):
    """Smooth blobs stretched to [lo, hi]: regions below, inside and above
    the domains tested here."""
    f = inputs.blob_field(dims, inputs.blob_params(5, dims, seed, sigma_range=(0.2, 0.4))).numpy().astype(np.float64)
    f = (f - f.min()) / max(f.max() - f.min(), 1e-12)
    return (lo + (hi - lo) * f).astype(np.float32)


def _brute_pixel(orc, field64, tf, cam, W, H, px, py, step, sm, sp, vmin, vmax):
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
        return np.zeros(4), np.zeros(0)
    dt = step * sp
    ts = []
    j = 0
    while te + (j + 0.5) * dt < tx:
        ts.append(te + (j + 0.5) * dt)
        j += 1
    if not ts:
        return np.zeros(4), np.zeros(0)
    q = (o[None, :] + np.array(ts)[:, None] * d[None, :]) / sp
    q = np.clip(q, 0, np.array(dims) - 1)
    s = map_coordinates(field64, [q[:, 2], q[:, 1], q[:, 0]], order=1, mode="nearest")
    knots_s = vmin + np.arange(tf.shape[0]) * ((vmax - vmin) / (tf.shape[0] - 1))
    rgba = np.stack([np.interp(s, knots_s, tf[:, c].astype(np.float64)) for c in range(4)], -1)
    alpha = 1 - np.exp(-sm * rgba[:, 3] * dt)
    C = np.zeros(3)
    for i in range(len(ts)):
        trans = 1.0
        for k in range(i):
            trans *= 1 - alpha[k]
        C += alpha[i] * rgba[i, :3] * trans
    A = 1 - np.prod(1 - alpha)
    return np.concatenate([C, [A]]), s


def _brute_check(orc, case, vmin, vmax):
    """Max abs difference of render_full / render_bricks from the brute
    force, and how many samples fell below, inside and above the domain."""
    g = np.random.default_rng(300 + case)
    dims = [(6, 5, 7), (7, 7, 6)][case % 2]
    w = vmax - vmin
    field = g.uniform(vmin - 0.8 * w, vmax + 0.8 * w, dims[::-1]).astype(np.float32)
    tf = inputs.make_tf(seed=11 + case)
    cams = [inputs.camera_from_direction(dims, (1, 0.7, 0.5)), inputs.random_cameras(dims, 1, seed=case)[0]]
    W, H = 7, 6
    sp = 1.0 / (max(dims) - 1)
    step, sm = 0.41, 7.0
    fr = orc.Frame(W, H, step_voxels=step, sigma_max=sm)
    part = inputs.regular_partition(dims, (2, 2, 1))
    bricks = orc.make_bricks(field, part, orc.F32)
    err = 0.0
    counts = np.zeros(3, np.int64)
    for cam in cams:
        full = orc.render_full(field, tf, cam, fr, vmin=vmin, vmax=vmax)
        br = orc.render_bricks(dims, bricks, tf, cam, fr, vmin=vmin, vmax=vmax)
        for p in range(W * H):
            ref, s = _brute_pixel(orc, field.astype(np.float64), tf, cam, W, H, p % W, p // W, step, sm, sp, vmin,
                                  vmax)
            assert full["nsamples"][p] == len(s)
            err = max(err, float(np.abs(full["rgba"][p] - ref).max()), float(np.abs(br["rgba"][p] - ref).max()))
            counts += [(s < vmin).sum(), ((s >= vmin) & (s <= vmax)).sum(), (s > vmax).sum()]
    return err, counts


@pytest.mark.parametrize("case", [0, 1])
@pytest.mark.parametrize("domain", DOMAINS)
def test_brute_force_non_unit_domain(orc, case, domain):
    err, counts = _brute_check(orc, case, *domain)
    # the field crosses both ends: each side of the clamp is exercised
    assert counts.min() > 20, counts
    assert err <= 1e-13, err


# --------------------------------------------------------------------------
# gradients on both clamped sides
# --------------------------------------------------------------------------

def _grad_problem(domain, seed=3, dims=(14, 12, 10)):
    w = domain[1] - domain[0]
    f = _field(dims, seed, domain[0] - 0.5 * w, domain[1] + 0.5 * w)
    tf = inputs.make_tf(seed=91 + seed)
    part = inputs.regular_partition(dims, (2, 1, 2))
    cam = inputs.camera_from_direction(dims, (1, 0.6, 0.45))
    W, H = 11, 9
    g = np.random.default_rng(seed).normal(size=(W * H, 4))
    return dims, f, tf, part, cam, W, H, g


def _loss(orc, dims, f, tf, part, cam, fr, g, vmin, vmax):
    br = orc.render_bricks(dims, orc.make_bricks(f, part, orc.F32), tf, cam, fr, vmin=vmin, vmax=vmax)
    return float(np.sum(br["rgba"] * g))


def _neighbourhood(f, z, y, x):
    """Values of the nodes sharing a cell with node (z, y, x): every sample
    the node's value reaches interpolates only these."""
    return f[max(z - 1, 0):z + 2, max(y - 1, 0):y + 2, max(x - 1, 0):x + 2]


def _voxel_picks(f, dvol, vmin, vmax, eps, n_each=6, seed=0):
    """Voxels whose whole neighbourhood lies below vmin - eps, above vmax +
    eps, or inside (vmin + 2 eps, vmax - 2 eps) with a non-zero gradient."""
    rng = np.random.default_rng(seed)
    below, above, inside = [], [], []
    for z, y, x in np.ndindex(*f.shape):
        nb = _neighbourhood(f, z, y, x)
        if nb.max() < vmin - 2 * eps:
            below.append((z, y, x))
        elif nb.min() > vmax + 2 * eps:
            above.append((z, y, x))
        elif nb.min() > vmin + 2 * eps and nb.max() < vmax - 2 * eps and abs(dvol[z, y, x]) > 1e-3 * np.abs(dvol).max():
            inside.append((z, y, x))
    pick = lambda L: [L[i] for i in rng.choice(len(L), size=min(n_each, len(L)), replace=False)] if L else []
    return pick(below), pick(above), pick(inside)


def _fd_voxel(orc, prob, fr, vmin, vmax, z, y, x, eps):
    dims, f, tf, part, cam, W, H, g = prob
    f1 = f.copy(); f1[z, y, x] += eps
    f0 = f.copy(); f0[z, y, x] -= eps
    h = np.float64(f1[z, y, x]) - np.float64(f0[z, y, x])
    return (_loss(orc, dims, f1, tf, part, cam, fr, g, vmin, vmax) -
            _loss(orc, dims, f0, tf, part, cam, fr, g, vmin, vmax)) / h


@pytest.mark.parametrize("domain", DOMAINS)
def test_voxel_gradient_clamped_sides_match_fd(orc, domain):
    vmin, vmax = domain
    prob = _grad_problem(domain)
    dims, f, tf, part, cam, W, H, g = prob
    fr = orc.Frame(W, H, sigma_max=16.0)
    _, dvol = orc.grad_bricks(dims, orc.make_bricks(f, part, orc.F32), tf, cam, fr, g, vmin=vmin, vmax=vmax)
    eps = np.float32(1e-4)
    below, above, inside = _voxel_picks(f, dvol, vmin, vmax, eps)
    assert len(below) >= 3 and len(above) >= 3 and len(inside) >= 3, (len(below), len(above), len(inside))
    gmax = np.abs(dvol).max()
    assert gmax > 0
    for (z, y, x) in below + above:
        # every sample the voxel reaches is clamped: no change, no gradient
        assert dvol[z, y, x] == 0.0
        assert _fd_voxel(orc, prob, fr, vmin, vmax, z, y, x, eps) == 0.0
    for (z, y, x) in inside:
        fd = _fd_voxel(orc, prob, fr, vmin, vmax, z, y, x, eps)
        assert abs(fd - dvol[z, y, x]) <= 1e-6 * gmax + 1e-4 * abs(fd), ((z, y, x), fd, dvol[z, y, x])


@pytest.mark.parametrize("domain", DOMAINS)
def test_tf_end_entries_match_fd(orc, domain):
    """The clamped samples weigh fully on the first or the last entry: the
    TF gradient there (and at interior entries) equals central differences."""
    vmin, vmax = domain
    prob = _grad_problem(domain, seed=4)
    dims, f, tf, part, cam, W, H, g = prob
    fr = orc.Frame(W, H, sigma_max=16.0)
    dtf, _ = orc.grad_bricks(dims, orc.make_bricks(f, part, orc.F32), tf, cam, fr, g, want_volume=False, vmin=vmin,
                             vmax=vmax)
    n = tf.shape[0]
    nz = [i for i in range(1, n - 1) if np.abs(dtf[i]).max() > 1e-3 * np.abs(dtf).max()]
    entries = [0, n - 1] + list(np.random.default_rng(2).choice(nz, size=min(6, len(nz)), replace=False))
    assert np.abs(dtf[0]).max() > 1e-3 * np.abs(dtf).max() and np.abs(dtf[n - 1]).max() > 1e-3 * np.abs(dtf).max()
    e = np.float32(1e-6)
    for i in entries:
        for c in range(4):
            t1 = tf.copy(); t1[i, c] += e
            t0 = tf.copy(); t0[i, c] -= e
            h = np.float64(t1[i, c]) - np.float64(t0[i, c])
            fd = (_loss(orc, dims, f, t1, part, cam, fr, g, vmin, vmax) -
                  _loss(orc, dims, f, t0, part, cam, fr, g, vmin, vmax)) / h
            assert abs(fd - dtf[i, c]) <= 1e-5 * abs(dtf).max() + 1e-4 * abs(fd), (i, c, fd, dtf[i, c])


# --------------------------------------------------------------------------
# planted mistakes (compiled into a copy of the oracle source)
# --------------------------------------------------------------------------

def _planted(orc, tmp_path, old, new, name):
    src = open(orc._SRC).read()
    assert src.count(old) == 1, "planting site not found exactly once: %r" % old
    path = os.path.join(str(tmp_path), name + ".c")
    with open(path, "w") as fh:
        fh.write(src.replace(old, new))
    return orc.compile_source(path, os.path.join(str(tmp_path), name + ".so"))


DOMAIN_LINE = "double x = (s - tf->vmin) / (tf->vmax - tf->vmin);"
CLAMP_LINE = "if (x < 0.0) { x = 0.0; d = 0.0; }"


def test_planted_domain_mistake_fails_brute_force(orc, tmp_path):
    """(s - vmin) (n - 1) / vmax instead of (s - vmin) (n - 1) / (vmax -
    vmin): invisible on [0, 1], caught by the brute force on a non-unit
    domain."""
    lib = _planted(orc, tmp_path, DOMAIN_LINE, "double x = (s - tf->vmin) / tf->vmax;", "plant_domain")
    err_ok, _ = _brute_check(orc, 0, 0.0, 1.0)
    assert err_ok <= 1e-13
    with orc.library(lib):
        err_unit, _ = _brute_check(orc, 0, 0.0, 1.0)
        err, _ = _brute_check(orc, 0, *DOMAINS[0])
    assert err_unit <= 1e-13          # the unit domain cannot see it
    assert err > 1e-3, err


def test_planted_unzeroed_derivative_fails_fd(orc, tmp_path):
    """du/ds kept on the lower clamped side: the oracle then reports a field
    gradient where central differences see none."""
    lib = _planted(orc, tmp_path, CLAMP_LINE, "if (x < 0.0) { x = 0.0; }", "plant_clamp")
    vmin, vmax = DOMAINS[0]
    prob = _grad_problem(DOMAINS[0])
    dims, f, tf, part, cam, W, H, g = prob
    fr = orc.Frame(W, H, sigma_max=16.0)
    _, dvol = orc.grad_bricks(dims, orc.make_bricks(f, part, orc.F32), tf, cam, fr, g, vmin=vmin, vmax=vmax)
    below, _, _ = _voxel_picks(f, dvol, vmin, vmax, np.float32(1e-4))
    with orc.library(lib):
        _, bad = orc.grad_bricks(dims, orc.make_bricks(f, part, orc.F32), tf, cam, fr, g, vmin=vmin, vmax=vmax)
    # the planted oracle reports gradients on voxels the FD test pins to zero
    assert max(abs(bad[v]) for v in below) > 1e-3 * np.abs(dvol).max()
