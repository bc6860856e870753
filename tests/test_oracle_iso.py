"""Oracle pins for the iso-surface fragments (first hit per brick, depth
composite).

* closed form: on a linear field (exact in float32 and in trilinear
  interpolation) the surface point of every hit lies on the plane
  s = iso, its normal is the field's gradient, so the shading factor is
  0.25 + 0.75 |d_x| / |d|;
* K-brick invariant: per-brick first hits (each brick testing the pairs
  whose later sample it owns, with its ghost layer) composited by smallest
  key reproduce the unpartitioned render exactly, regular and k-d
  partitions, cameras outside and inside;
* brute force: samples by scipy.ndimage.map_coordinates (order 1) along the
  ray, the first sign change found by numpy, the gradient by central
  differences inside the cell;
* planted mistake: bricks without ghost nodes break the invariant.
"""
import numpy as np
import pytest
from scipy import ndimage

from paper_2407_00179_b300 import inputs

PARTS = {
    "2x2x2": lambda d: inputs.regular_partition(d, (2, 2, 2)),
    "3x2x4": lambda d: inputs.regular_partition(d, (3, 2, 4)),
    "kd9": lambda d: inputs.kd_partition(d, 9, seed=5),
}


def _blobs(dims, seed=0):
    return inputs.blob_field(dims, inputs.blob_params(8, dims, seed, sigma_range=(0.15, 0.3))).numpy()


def test_linear_field_closed_form(orc):
    dims = (33, 21, 17)
    x = np.arange(dims[0], dtype=np.float64)
    f = np.broadcast_to((x / 32.0)[None, None, :], (dims[2], dims[1], dims[0])).astype(np.float32)
    iso = 0.421875                              # 13.5/32: the plane x = 13.5, mid-cell
    tf = inputs.make_tf(1234)
    fr = orc.Frame(61, 47, step_voxels=0.5)
    checked = 0
    for cam in inputs.random_cameras(dims, 3, seed=2):
        r = orc.render_iso(dims, tf, cam, fr, iso, field=f)
        hit = r["key"] >= 0
        sp = 1.0 / (max(dims) - 1)
        tfv = np.array([np.interp(iso, np.linspace(0, 1, len(tf)), tf[:, c].astype(np.float64)) for c in range(3)])
        for k in np.nonzero(hit & ((r["flags"] & orc.FLAG_ISO_AMBIG) == 0))[0]:
            px, py = k % fr.width, k // fr.width
            o, d = orc.camera_ray(cam, fr.width, fr.height, px, py)
            p = np.asarray(o) + r["depth"][k] * np.asarray(d)
            # the surface point is on the plane x / 32 = iso (node units)
            assert abs((p[0] / sp) / 32.0 - iso) < 1e-12
            fac = 0.25 + 0.75 * abs(d[0]) / np.linalg.norm(d)
            np.testing.assert_allclose(r["rgba"][k, :3], tfv * fac, rtol=0, atol=1e-12)
            assert r["rgba"][k, 3] == 1.0
            checked += 1
        assert np.all(np.isinf(r["depth"][~hit])) and np.all(r["rgba"][~hit] == 0.0)
    assert checked > 100


@pytest.mark.parametrize("pname", list(PARTS))
@pytest.mark.parametrize("inside", [False, True])
def test_kbrick_equals_unpartitioned(orc, pname, inside):
    dims = (24, 20, 28)
    f = _blobs(dims, 1)
    tf = inputs.make_tf(1234)
    bricks = orc.make_bricks(f, PARTS[pname](dims), orc.F32)
    fr = orc.Frame(29, 21, step_voxels=0.5)
    hits = []
    for iso in (0.3, 0.55):
        for cam in inputs.random_cameras(dims, 2, seed=7 + list(PARTS).index(pname), inside=inside):
            a = orc.render_iso(dims, tf, cam, fr, iso, field=f)
            b = orc.render_iso(dims, tf, cam, fr, iso, bricks=bricks)
            np.testing.assert_array_equal(a["key"], b["key"])
            np.testing.assert_array_equal(a["rgba"], b["rgba"])
            np.testing.assert_array_equal(a["depth"], b["depth"])
            # the composited key is the smallest per-brick key
            fk = b["frag_key"].astype(np.int64)
            m = fk.min(axis=1)
            np.testing.assert_array_equal(np.where(m == 2 ** 31 - 1, -1, m), b["key"])
            hits.append((a["key"] >= 0).mean())
    assert np.mean(hits) > 0.02


def test_brute_force(orc):
    dims = (12, 10, 11)
    f = _blobs(dims, 4)
    tf = inputs.make_tf(77)
    iso = 0.35
    fr = orc.Frame(17, 13, step_voxels=0.5)
    sp = 1.0 / (max(dims) - 1)
    cam = inputs.camera_from_direction(dims, (0.8, -0.5, 0.6))
    r = orc.render_iso(dims, tf, cam, fr, iso, field=f)
    lo = np.zeros(3)
    hi = (np.array(dims) - 1) * sp
    n_hit = 0

    def value(q):      # q in node units (x, y, z)
        return ndimage.map_coordinates(f.astype(np.float64), [[q[2]], [q[1]], [q[0]]], order=1)[0]

    for k in range(fr.width * fr.height):
        px, py = k % fr.width, k // fr.width
        o, d = np.array(orc.camera_ray(cam, fr.width, fr.height, px, py)[0]), np.array(
            orc.camera_ray(cam, fr.width, fr.height, px, py)[1])
        with np.errstate(divide="ignore", invalid="ignore"):
            t0, t1 = (lo - o) / d, (hi - o) / d
        te = max(0.0, np.nanmax(np.minimum(t0, t1)))
        tx = np.nanmin(np.maximum(t0, t1))
        dt = 0.5 * sp
        js = np.arange(0, int(np.ceil((tx - te) / dt)) + 2)
        ts = te + (js + 0.5) * dt
        ts = ts[ts < tx]
        if r["flags"][k] & orc.FLAG_ISO_AMBIG:
            continue
        if tx <= te or len(ts) < 2:
            assert r["key"][k] == -1
            continue
        qs = [np.clip((o + t * d - lo) / sp, 0, np.array(dims) - 1) for t in ts]
        s = np.array([value(q) for q in qs])
        above = s >= iso
        ch = np.nonzero(above[1:] != above[:-1])[0]
        if len(ch) == 0:
            assert r["key"][k] == -1
            continue
        h = ch[0] + 1
        assert r["key"][k] == h
        fh = (iso - s[h - 1]) / (s[h] - s[h - 1])
        assert abs(r["depth"][k] - (ts[h - 1] + fh * dt)) < 1e-12
        # shading from central differences of the interpolant inside the cell
        q = np.clip((o + r["depth"][k] * d - lo) / sp, 0, np.array(dims) - 1)
        e = 1e-7
        g = np.array([(value(q + e * u) - value(q - e * u)) / (2 * e) for u in np.eye(3)])
        fac = 0.25 + 0.75 * abs(g @ d) / (np.linalg.norm(g) * np.linalg.norm(d))
        tfv = np.array([np.interp(iso, np.linspace(0, 1, len(tf)), tf[:, c].astype(np.float64)) for c in range(3)])
        np.testing.assert_allclose(r["rgba"][k, :3], tfv * fac, rtol=0, atol=1e-7)
        n_hit += 1
    assert n_hit > 20


def test_ghost_layer_is_needed(orc):
    """Planted mistake on the CPU: without ghost nodes a brick cannot
    evaluate the sample before its first one, and hits move."""
    dims = (24, 20, 28)
    f = _blobs(dims, 1)
    part = inputs.regular_partition(dims, (2, 2, 2))
    bricks = orc.make_bricks(f, part, orc.F32)
    for b in bricks:
        d = b.data.copy()
        for a, ax in ((0, 2), (1, 1), (2, 0)):
            for end, nxt in ((0, 1), (-1, -2)):
                if (end == 0 and b.lo[a] > 0) or (end == -1 and b.hi[a] < dims[a]):
                    sl = [slice(None)] * 3
                    sl[ax] = end
                    sl2 = list(sl)
                    sl2[ax] = nxt
                    d[tuple(sl)] = d[tuple(sl2)]
        b.data = d
    tf = inputs.make_tf(1234)
    fr = orc.Frame(29, 21)
    cam = inputs.camera_from_direction(dims, (1, 0.7, 0.5))
    a = orc.render_iso(dims, tf, cam, fr, 0.3, field=f)
    b = orc.render_iso(dims, tf, cam, fr, 0.3, bricks=bricks)
    both = np.isfinite(a["depth"]) & np.isfinite(b["depth"])
    bad = (a["key"] != b["key"]) | (both & (np.abs(np.where(both, a["depth"] - b["depth"], 0.0)) > 1e-9))
    assert bad.sum() > 0
