"""Oracle pins for deep fragments: empty-space skipping over macro-cells of
8^3 cells splits a brick's segment into one fragment per run of evaluated
samples (at most `deep` per brick and pixel), and the compositor sorts the
variable count per pixel.

* the deep composite equals the sort-last composite (1e-12; samples of a
  transparent macro-cell have alpha exactly 0 and over is associative), for
  several caps, regular and k-d partitions, early termination off and on;
  per brick, its deep fragments composited in key order equal its
  sort-last fragment (a wrong transmittance reset at a split fails this);
* the split itself against brute force written here with numpy: sample
  positions from the ray, owners from the owned boxes, macro-cell ranges
  from the stored nodes, transparency from the TF entries a range reads,
  runs of evaluated samples -> keys and counts;
* special cases: no transparent TF entry gives one fragment per brick equal
  to the sort-last one bit for bit; an all-transparent TF gives no fragment;
  cap 1 gives the sort-last fragment's RGBA bit for bit; depth never lies in
  front of the sort-last depth.
"""
import numpy as np
import pytest

from paper_2407_00179_b300 import inputs

DIMS = (40, 36, 44)
PARTS = {
    "2x2x2": lambda d: inputs.regular_partition(d, (2, 2, 2)),
    "kd7": lambda d: inputs.kd_partition(d, 7, seed=3),
}

def _setup(cut=0.35, seed=1):
    f = inputs.blob_field(DIMS, inputs.blob_params(10, DIMS, seed)).numpy()
    return f, inputs.make_tf(1234, transparent_below=cut)


def _amb(orc):
    return orc.FLAG_EXIT_AMBIG | orc.FLAG_OWNER_AMBIG | orc.FLAG_MACRO_AMBIG | orc.FLAG_ERT_AMBIG


@pytest.mark.parametrize("pname", list(PARTS))
@pytest.mark.parametrize("ert", [0.0, 0.9])
def test_deep_composite_equals_sort_last(orc, pname, ert):
    f, tf = _setup()
    bricks = orc.make_bricks(f, PARTS[pname](DIMS), orc.F32)
    fr = orc.Frame(31, 27, step_voxels=0.5, sigma_max=40.0, ert=ert)
    split = 0
    for cam in inputs.random_cameras(DIMS, 2, seed=21):
        ref = orc.render_bricks(DIMS, bricks, tf, cam, fr)
        for deep in (1, 2, 4, 16):
            d = orc.render_deep(DIMS, bricks, tf, cam, fr, deep=deep)
            assert np.abs(d["rgba"] - ref["rgba"]).max() <= 1e-12
            assert np.all(d["nsamples"] <= ref["nsamples"])
            fin = np.isfinite(ref["depth"])
            np.testing.assert_array_equal(np.isfinite(d["depth"]), fin)
            assert np.all(d["depth"][fin] >= ref["depth"][fin] - 1e-12)
            # per brick: its fragments in key order composite to its sort-last fragment
            for b in range(len(bricks)):
                keys = d["frag_key"][:, b, :]
                C = np.zeros((keys.shape[0], 4))
                for i in range(deep):            # fragments are stored in key order
                    live = keys[:, i] != 2 ** 31 - 1
                    C[live] += (1.0 - C[live, 3:4]) * d["frag_rgba"][live, b, i]
                    if i > 0:
                        both = live & (keys[:, i - 1] != 2 ** 31 - 1)
                        assert np.all(keys[both, i] > keys[both, i - 1])
                assert np.abs(C - ref["frag_rgba"][:, b]).max() <= 1e-12
            if deep == 16:
                split += int((d["frag_count"] > 1).sum())
                assert d["nsamples"].sum() < 0.9 * ref["nsamples"].sum()
        assert ref["rgba"][:, 3].max() > 0.2
    assert split > 10                                  # segments actually split


def _ray_box(o, d, lo, hi):
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        t0 = (lo - o) * inv
        t1 = (hi - o) * inv
    tmin = np.nanmax(np.minimum(t0, t1))
    tmax = np.nanmin(np.maximum(t0, t1))
    return max(tmin, 0.0), tmax


def _expected_split(orc, bricks, tf, cam, fr, px, py, deep):
    """Brute force: keys and counts per brick of one pixel's deep fragments."""
    sp = 1.0 / (max(DIMS) - 1)
    o, d = orc.camera_ray(cam, fr.width, fr.height, px, py)
    hi = (np.array(DIMS) - 1) * sp
    te, tx = _ray_box(o, d, np.zeros(3), hi)
    K = len(bricks)
    keys = [[] for _ in range(K)]
    if not te < tx:
        return keys
    dt = fr.step_voxels * sp
    n = int(np.floor((tx - te) / dt + 0.5))
    while n > 0 and te + (n - 0.5) * dt >= tx:
        n -= 1
    while te + (n + 0.5) * dt < tx:
        n += 1
    ntf = tf.shape[0]

    def i0(v):
        u = np.clip(v, 0.0, 1.0) * (ntf - 1)
        return min(int(np.floor(u)), ntf - 2)

    empty = []
    boxes = []
    for b in bricks:
        s_lo = np.maximum(np.array(b.lo) - 1, 0)
        s_hi = np.minimum(np.array(b.hi), np.array(DIMS) - 1)
        bn = s_hi - s_lo + 1
        v = b.data.astype(np.float64).reshape(bn[2], bn[1], bn[0]) * b.scale
        mn = (bn - 2) // 8 + 1
        e = np.zeros((mn[2], mn[1], mn[0]), bool)
        for mz in range(mn[2]):
            for my in range(mn[1]):
                for mx in range(mn[0]):
                    blk = v[8 * mz:8 * mz + 9, 8 * my:8 * my + 9, 8 * mx:8 * mx + 9]
                    e[mz, my, mx] = np.all(tf[i0(blk.min()):i0(blk.max()) + 2, 3] == 0.0)
        empty.append(e)
        boxes.append((s_lo, bn))
    run = [False] * K
    for j in range(n):
        q = np.clip((o + (te + (j + 0.5) * dt) * d) / sp, 0.0, np.array(DIMS) - 1.0)
        owner = -1
        for k, b in enumerate(bricks):
            r0 = np.maximum(np.array(b.lo) - 0.5, 0.0)
            r1 = np.minimum(np.array(b.hi) - 0.5, np.array(DIMS) - 1.0)
            closed = np.array(b.hi) >= np.array(DIMS)
            if np.all(q >= r0) and np.all(np.where(closed, q <= r1, q < r1)):
                owner = k
                break
        s_lo, bn = boxes[owner]
        c = np.clip(np.floor(q).astype(int), s_lo, s_lo + bn - 2) - s_lo
        if empty[owner][c[2] // 8, c[1] // 8, c[0] // 8]:
            run[owner] = False
            continue
        if not run[owner] and len(keys[owner]) < deep:
            keys[owner].append(j)
        run[owner] = True
    return keys


@pytest.mark.parametrize("deep", [2, 4])
def test_split_against_brute_force(orc, deep):
    f, tf = _setup()
    bricks = orc.make_bricks(f, PARTS["kd7"](DIMS), orc.F32)
    fr = orc.Frame(31, 27, step_voxels=0.5, sigma_max=20.0)
    cam = inputs.random_cameras(DIMS, 2, seed=21)[1]
    # every pixel whose segments split, and as many others
    full = orc.render_deep(DIMS, bricks, tf, cam, fr, deep=deep)
    many = np.flatnonzero(full["frag_count"].max(axis=1) > 1)
    rng = np.random.default_rng(0)
    pix = np.concatenate([many, rng.choice(fr.width * fr.height, 40, replace=False)]).astype(np.int32)
    d = orc.render_deep(DIMS, bricks, tf, cam, fr, deep=deep, pix=pix)
    checked = multi = 0
    for k, p in enumerate(pix):
        if d["flags"][k] & _amb(orc):
            continue
        exp = _expected_split(orc, bricks, tf, cam, fr, int(p % fr.width), int(p // fr.width), deep)
        for b in range(len(bricks)):
            got = [int(x) for x in d["frag_key"][k, b] if x != 2 ** 31 - 1]
            assert got == exp[b], (int(p), b, got, exp[b])
            assert d["frag_count"][k, b] == len(exp[b])
            multi += len(exp[b]) > 1
        checked += 1
    assert checked > 40 and multi > 5


def test_special_cases(orc):
    f, tf = _setup()
    bricks = orc.make_bricks(f, PARTS["2x2x2"](DIMS), orc.F32)
    fr = orc.Frame(21, 17, step_voxels=0.5, sigma_max=30.0, ert=0.95)
    cam = inputs.camera_from_direction(DIMS, (1.0, 0.6, 0.4))
    # no transparent entry: one fragment per brick, the sort-last one exactly
    opaque = inputs.make_tf(1234)
    opaque[:, 3] = np.maximum(opaque[:, 3], np.float32(1e-3))
    ref = orc.render_bricks(DIMS, bricks, opaque, cam, fr)
    d = orc.render_deep(DIMS, bricks, opaque, cam, fr, deep=4)
    np.testing.assert_array_equal(d["frag_key"][:, :, 0], ref["frag_key"])
    np.testing.assert_array_equal(d["frag_rgba"][:, :, 0], ref["frag_rgba"])
    assert np.all(d["frag_count"] == (ref["frag_key"] != 2 ** 31 - 1))
    np.testing.assert_array_equal(d["nsamples"], ref["nsamples"])
    # all entries transparent: nothing is evaluated
    clear = tf.copy()
    clear[:, 3] = 0.0
    d = orc.render_deep(DIMS, bricks, clear, cam, fr, deep=4)
    assert d["nsamples"].sum() == 0 and np.all(d["frag_count"] == 0)
    assert np.all(d["rgba"] == 0.0) and np.all(np.isinf(d["depth"]))
    # cap 1: the sort-last fragment's RGBA, keys at the first evaluated sample
    ref = orc.render_bricks(DIMS, bricks, tf, cam, fr)
    d = orc.render_deep(DIMS, bricks, tf, cam, fr, deep=1)
    live = d["frag_key"][:, :, 0] != 2 ** 31 - 1
    np.testing.assert_array_equal(d["frag_rgba"][:, :, 0][live], ref["frag_rgba"][live])
    assert np.all(d["frag_key"][:, :, 0][live] >= ref["frag_key"][live])
    assert np.all(ref["frag_rgba"][~live] == 0.0)
