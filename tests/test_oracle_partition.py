"""Oracle pins for the partitioned (data-parallel) path.

* K-brick invariant: per-brick fragments with a one-node ghost layer,
  composited in key order, reproduce the unpartitioned render (FP64, 1e-12),
  for regular and uneven k-d partitions, cameras outside and inside the
  volume (sort-last compositing is exact for convex parts, §2.1);
* compositing: K = 1 is the identity, "over" is associative, empty
  fragments are skipped;
* order: ascending fragment keys equal the k-d front-to-back order seen from
  the eye, restricted to the bricks the ray actually crosses (§5.1.1: sorting
  by depth needs no a-priori compositing order).
"""
import numpy as np
import pytest

from paper_2407_00179_b300 import inputs


def _setup(dims=(24, 20, 28), seed=0):
    f = inputs.blob_field(dims, inputs.blob_params(8, dims, seed)).numpy()
    tf = inputs.make_tf(seed=1234)
    return f, tf


PARTS = {
    "2x1x1": lambda d: inputs.regular_partition(d, (2, 1, 1)),
    "2x2x2": lambda d: inputs.regular_partition(d, (2, 2, 2)),
    "3x2x4": lambda d: inputs.regular_partition(d, (3, 2, 4)),
    "kd7": lambda d: inputs.kd_partition(d, 7, seed=3),
    "kd13": lambda d: inputs.kd_partition(d, 13, seed=9),
}


@pytest.mark.parametrize("pname", list(PARTS))
@pytest.mark.parametrize("inside", [False, True])
def test_kbrick_equals_unpartitioned(orc, pname, inside):
    dims = (24, 20, 28)
    f, tf = _setup(dims)
    part = PARTS[pname](dims)
    bricks = orc.make_bricks(f, part, orc.F32)
    W, H = 23, 19
    fr = orc.Frame(W, H, step_voxels=0.5, sigma_max=8.0)
    for cam in inputs.random_cameras(dims, 2, seed=list(PARTS).index(pname), inside=inside):
        full = orc.render_full(f, tf, cam, fr)
        br = orc.render_bricks(dims, bricks, tf, cam, fr)
        assert np.abs(br["rgba"] - full["rgba"]).max() <= 1e-12
        np.testing.assert_array_equal(br["nsamples"], full["nsamples"])
        assert full["rgba"][:, 3].max() > 0.05          # the image is not empty


def test_kbrick_invariant_f16_storage(orc):
    """f16 and bf16 storage use scale 1, so quantising node by node commutes
    with partitioning: the partitioned render of quantised bricks equals the
    unpartitioned render of the quantised global field."""
    dims = (24, 20, 28)
    f, tf = _setup(dims, seed=2)
    part = PARTS["kd7"](dims)
    fr = orc.Frame(17, 13)
    cam = inputs.camera_from_direction(dims, (0.3, -1, 0.4))
    for dt in (orc.F16, orc.BF16):
        bricks = orc.make_bricks(f, part, dt)
        fq = orc.dequantize(orc.quantize(f, dt), dt).astype(np.float32)
        full = orc.render_full(fq, tf, cam, fr)
        br = orc.render_bricks(dims, bricks, tf, cam, fr)
        assert np.abs(br["rgba"] - full["rgba"]).max() <= 1e-12


def test_ghost_layer_is_needed(orc):
    """Planted mistake on the CPU: bricks without ghost nodes (cell index
    clamped inside the owned nodes) break the invariant near brick faces."""
    dims = (24, 20, 28)
    f, tf = _setup(dims)
    part = PARTS["2x2x2"](dims)
    bricks = orc.make_bricks(f, part, orc.F32)
    # overwrite each brick's ghost nodes with the nearest owned node
    for b in bricks:
        s_lo, s_n = orc.stored_box(dims, b.lo, b.hi)
        d = b.data.copy()
        for a, ax in ((0, 2), (1, 1), (2, 0)):
            if b.lo[a] > 0:
                sl = [slice(None)] * 3
                sl[ax] = 0
                sl2 = list(sl)
                sl2[ax] = 1
                d[tuple(sl)] = d[tuple(sl2)]
            if b.hi[a] < dims[a]:
                sl = [slice(None)] * 3
                sl[ax] = -1
                sl2 = list(sl)
                sl2[ax] = -2
                d[tuple(sl)] = d[tuple(sl2)]
        b.data = d
    fr = orc.Frame(23, 19)
    cam = inputs.camera_from_direction(dims, (1, 0.7, 0.5))
    full = orc.render_full(f, tf, cam, fr)
    br = orc.render_bricks(dims, bricks, tf, cam, fr)
    assert np.abs(br["rgba"] - full["rgba"]).max() > 1e-4


def test_composite_identity_and_empty(orc):
    g = np.random.default_rng(5)
    n = 500
    fr = g.uniform(0, 1, (n, 1, 4))
    fr[:, :, :3] *= fr[:, :, 3:]          # premultiplied
    key = g.integers(0, 1000, (n, 1)).astype(np.int32)
    key[::7] = orc.KEY_EMPTY
    rgba, order = orc.composite(fr, key)
    ne = key[:, 0] != orc.KEY_EMPTY
    np.testing.assert_array_equal(rgba[ne], fr[ne, 0])              # bit-exact identity
    np.testing.assert_array_equal(rgba[~ne], 0.0)
    np.testing.assert_array_equal(order[ne, 0], 0)
    np.testing.assert_array_equal(order[~ne, 0], 0xFF)


def test_composite_associative_and_sorted(orc):
    g = np.random.default_rng(6)
    n = 300
    frs = g.uniform(0, 1, (n, 3, 4))
    frs[..., :3] *= frs[..., 3:]
    keys = np.stack([g.permutation(3) * 10 for _ in range(n)]).astype(np.int32)
    full, order = orc.composite(frs, keys)
    # the order is the key order
    np.testing.assert_array_equal(order, np.argsort(keys, axis=1))
    srt = np.take_along_axis(frs, np.argsort(keys, axis=1)[..., None], axis=1)
    a, b, c = srt[:, 0], srt[:, 1], srt[:, 2]
    k2 = np.tile(np.array([0, 1], np.int32), (n, 1))
    ab, _ = orc.composite(np.stack([a, b], 1), k2)
    bc, _ = orc.composite(np.stack([b, c], 1), k2)
    left, _ = orc.composite(np.stack([ab, c], 1), k2)
    right, _ = orc.composite(np.stack([a, bc], 1), k2)
    assert np.abs(left - right).max() < 1e-15
    assert np.abs(left - full).max() < 1e-15
    # reordering the input slots does not change the result
    perm = g.permutation(3)
    full2, _ = orc.composite(frs[:, perm], keys[:, perm])
    np.testing.assert_array_equal(full, full2)


@pytest.mark.parametrize("pname", ["2x2x2", "3x2x4", "kd13"])
@pytest.mark.parametrize("inside", [False, True])
def test_key_order_is_kd_eye_order(orc, pname, inside):
    dims = (24, 20, 28)
    f, tf = _setup(dims)
    part = PARTS[pname](dims)
    bricks = orc.make_bricks(f, part, orc.F32)
    W, H = 31, 27
    fr = orc.Frame(W, H)
    sp = 1.0 / (max(dims) - 1)
    nonempty_multi = 0
    for cam in inputs.random_cameras(dims, 2, seed=11, inside=inside):
        br = orc.render_bricks(dims, bricks, tf, cam, fr)
        kd = list(orc.kd_order(part, np.array(cam.eye) / sp))
        assert sorted(kd) == list(range(part.num_ranks))
        for p in range(W * H):
            keys = br["frag_key"][p]
            ne = [k for k in range(part.num_ranks) if keys[k] != orc.KEY_EMPTY]
            expect = [k for k in kd if k in ne]
            got = [int(x) for x in br["order"][p] if x != 0xFF]
            assert got == expect
            nonempty_multi += len(ne) > 1
    assert nonempty_multi > 50


def test_order_rejects_wrong_tree(orc):
    """Planted mistake on the CPU: visiting the far child first gives the
    reverse order, which the key order contradicts."""
    dims = (24, 20, 28)
    part = PARTS["2x1x1"](dims)
    sp = 1.0 / (max(dims) - 1)
    cam = inputs.camera_from_direction(dims, (1, 0.1, 0.1))     # eye on the +x side
    kd = list(orc.kd_order(part, np.array(cam.eye) / sp))
    assert kd == [1, 0]
    flipped = inputs.Partition(part.lo, part.hi, part.axis, part.split, part.right, part.left)
    wrong = list(orc.kd_order(flipped, np.array(cam.eye) / sp))
    assert wrong == [0, 1]
    f, tf = _setup(dims)
    br = orc.render_bricks(dims, orc.make_bricks(f, part, orc.F32), tf, cam, orc.Frame(9, 9))
    both = [p for p in range(81) if np.all(br["frag_key"][p] != orc.KEY_EMPTY)]
    assert both and all(list(br["order"][p]) == kd != wrong for p in both)


def test_ert_is_per_fragment(orc):
    """Early termination stops a brick's own accumulation once its local
    opacity passes the threshold; bricks behind are still marched."""
    dims = (24, 20, 28)
    f, tf = _setup(dims)
    tf = tf.copy()
    tf[:, 3] = np.maximum(tf[:, 3], 0.8)
    part = PARTS["2x1x1"](dims)
    bricks = orc.make_bricks(f, part, orc.F32)
    cam = inputs.camera_from_direction(dims, (1, 0.05, 0.02))
    fr0 = orc.Frame(15, 15, sigma_max=40.0)
    fr1 = orc.Frame(15, 15, sigma_max=40.0, ert=0.9)
    a = orc.render_bricks(dims, bricks, tf, cam, fr0)
    b = orc.render_bricks(dims, bricks, tf, cam, fr1)
    stopped = b["frag_nsamp"] < a["frag_nsamp"]
    assert stopped.sum() > 10
    fa = b["frag_rgba"][..., 3]
    assert np.all(fa[stopped] > 0.9)
    # a stopped fragment is the prefix of the full one: its opacity never
    # exceeds the full opacity and the next-to-last state is below threshold
    assert np.all(fa <= a["frag_rgba"][..., 3] + 1e-15)
    assert np.all(b["frag_nsamp"][~stopped] == a["frag_nsamp"][~stopped])
    assert np.all(b["nsamples"] <= a["nsamples"])
