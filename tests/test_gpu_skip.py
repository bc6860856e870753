"""GPU empty-space skipping (DPV_FRAME_SKIP) in the forward march.

A sample whose TF opacity is exactly 0 leaves the colour and transmittance
unchanged (the emission-absorption step of §5.1.1 with alpha = 0), so
skipping the samples of macro-cells that can only reach transparent TF
entries changes no bit of the result.  The checks:

* frames and every rank's fragments (RGBA and key) bit-identical to the
  same frame without skipping: regular and k-d partitions, f32 / f16 /
  fp8 storage (per-brick scales), a camera inside, per-fragment early
  termination, the ordered march, all three gather layouts;
* fewer evaluated samples (the count drops by at least a quarter on a TF
  that hides the values below 0.35);
* the frame equals the FP64 oracle within 1e-5 (unflagged pixels);
* degenerate TFs: all entries transparent gives an empty frame with no
  sample evaluated; no transparent entry evaluates every sample;
* a new TF between renders reclassifies (matches a fresh non-skipping
  device), and so does a re-committed brick;
* the adjoint after a skipping forward equals the adjoint after a full one
  (it replays every sample: dalpha/dTF is not 0 where alpha is);
* the iso-surface, staged and allocation-free forms refuse the flag.
"""
import numpy as np
import pytest
import torch

from paper_2407_00179_b300 import build, dpv, inputs

import scenes

pytestmark = pytest.mark.gpu

TOL = 1e-5
CUT = 0.35

CASES = [
    dict(dims=(48, 40, 44), splits=(2, 2, 2), width=96, height=80),
    dict(dims=(50, 42, 36), kd=9, width=67, height=45, tile=(8, 4), storage="f16"),
    dict(dims=(50, 42, 36), kd=5, width=61, height=47, tile=(32, 8), inside=True),
    dict(dims=(40, 36, 32), splits=(2, 1, 2), width=52, height=44, storage="fp8", sigma_max=40.0, ert=0.95),
    dict(dims=(70, 38, 42), splits=(3, 1, 2), width=64, height=48, storage="bf16"),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    dpv.load()


def _scene(i, cut=CUT):
    c = dict(CASES[i])
    inside = c.pop("inside", False)
    dims = c.pop("dims")
    cams = inputs.random_cameras(dims, 2, seed=80 + i, inside=inside)
    sc = scenes.make(dims, cams=cams, nblobs=10, seed=i, **c)
    sc.tf = inputs.make_tf(1234, transparent_below=cut)
    return sc


def _device(sc, skip, gather="auto", ordered=False):
    dev = scenes.gpu_device(sc, order=False)
    dev.set_frame(sc.width, sc.height, step_voxels=sc.step, sigma_max=sc.sigma_max, ert=sc.ert, tile=sc.tile,
                  gather=gather, ordered=ordered, skip=skip)
    dev.reset_stats()
    dev.render()
    return dev


def _everything(dev, sc, fragments=True):
    out = []
    for c in range(len(sc.cams)):
        out += [t.clone() for t in dev.map_frame(c)]
        if fragments:
            for k in range(sc.part.num_ranks):
                out += [t.clone() for t in dev.read_fragments(c, k)]
    return out


def _assert_identical(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


@pytest.mark.parametrize("i", range(len(CASES)))
def test_skip_bit_identical_and_fewer_samples(i):
    sc = _scene(i)
    a = _device(sc, skip=True)
    b = _device(sc, skip=False)
    assert a.stats()["error_flags"] == 0
    _assert_identical(_everything(a, sc), _everything(b, sc))
    na, nb = a.stats()["samples_forward"], b.stats()["samples_forward"]
    print("case %d: %d of %d samples evaluated (%.2f)" % (i, na, nb, na / nb))
    assert 0 < na < 0.75 * nb
    a.release()
    b.release()


@pytest.mark.parametrize("gather", ["cell", "quad", "linear"])
@pytest.mark.parametrize("ordered", [False, True])
def test_skip_layouts_and_ordered(gather, ordered):
    sc = _scene(1)
    sc.sigma_max, sc.ert = 60.0, 0.95
    a = _device(sc, skip=True, gather=gather, ordered=ordered)
    b = _device(sc, skip=False, gather=gather, ordered=ordered)
    _assert_identical(_everything(a, sc, fragments=not ordered), _everything(b, sc, fragments=not ordered))
    assert a.stats()["samples_forward"] < b.stats()["samples_forward"]
    a.release()
    b.release()


def test_skip_axis_aligned_views():
    """Rays (nearly) parallel to a grid axis: their step along the other
    axes is tiny, where a jump over a macro-cell relies on its margin."""
    sc = _scene(0)
    sc.cams = [scenes.f32_camera(inputs.camera_from_direction(sc.dims, d))
               for d in ((1.0, 0.0, 0.0), (0.0, -1.0, 0.0), (0.0, 0.0, 1.0), (1.0, 1.0, 0.0))]
    a = _device(sc, skip=True)
    b = _device(sc, skip=False)
    _assert_identical(_everything(a, sc), _everything(b, sc))
    assert a.stats()["samples_forward"] < b.stats()["samples_forward"]
    a.release()
    b.release()


def test_skip_matches_fp64_oracle(orc):
    sc = _scene(0)
    dev = _device(sc, skip=True)
    bricks = scenes.oracle_bricks(orc, sc)
    for ci, cam in enumerate(sc.cams):
        ref = orc.render_bricks(sc.dims, bricks, sc.tf, cam, scenes.oracle_frame(orc, sc), spacing=sc.spacing)
        rgba, _ = dev.map_frame(ci)
        rgba = rgba.reshape(-1, 4).double().cpu().numpy()
        ok = (ref["flags"] & scenes.FLAG["exit"]) == 0
        assert ok.mean() > 0.9
        assert np.abs(rgba - ref["rgba"])[ok].max() <= TOL
        assert ref["rgba"][:, 3].max() > 0.2
    dev.release()


def test_degenerate_tables():
    sc = _scene(0)
    # every entry transparent: nothing to evaluate, an empty frame
    sc.tf = inputs.make_tf(1234, transparent_below=1.0)
    assert np.all(sc.tf[:, 3] == 0.0)
    a = _device(sc, skip=True)
    assert a.stats()["samples_forward"] == 0
    for c in range(len(sc.cams)):
        rgba, _ = a.map_frame(c)
        assert float(rgba.abs().max()) == 0.0
    a.release()
    # no transparent entry: every sample is evaluated
    sc.tf = inputs.make_tf(1234)
    sc.tf[:, 3] = np.maximum(sc.tf[:, 3], np.float32(1e-3))
    a = _device(sc, skip=True)
    b = _device(sc, skip=False)
    assert a.stats()["samples_forward"] == b.stats()["samples_forward"]
    _assert_identical(_everything(a, sc), _everything(b, sc))
    a.release()
    b.release()


def test_reclassified_after_new_tf_and_recommit():
    sc = _scene(2)
    a = _device(sc, skip=True)
    # a table transparent above 0.3 instead: the low-valued macro-cells
    # skipped so far are opaque now (a stale classification drops them)
    tf2 = inputs.make_tf(99)
    tf2[np.arange(tf2.shape[0]) >= int(0.3 * (tf2.shape[0] - 1)), 3] = 0.0
    a.set_tf(torch.from_numpy(tf2).cuda())
    a.reset_stats()
    a.render()
    sc2 = _scene(2)
    sc2.tf = tf2
    b = _device(sc2, skip=False)
    _assert_identical(_everything(a, sc2), _everything(b, sc2))
    assert a.stats()["samples_forward"] <= b.stats()["samples_forward"]
    b.release()
    # re-commit rank 0 with the field shifted up by 0.3: its ranges are rebuilt
    f3 = sc.field + np.float32(0.3)
    lo, hi = sc.part.lo[0], sc.part.hi[0]
    a.commit_brick(0, lo, hi, torch.from_numpy(f3).cuda(), sc.storage)
    a.render()
    c = scenes.gpu_device(sc2, order=False)
    c.commit_brick(0, lo, hi, torch.from_numpy(f3).cuda(), sc.storage)
    c.set_frame(sc.width, sc.height, step_voxels=sc.step, sigma_max=sc.sigma_max, ert=sc.ert, tile=sc.tile)
    c.render()
    _assert_identical(_everything(a, sc2), _everything(c, sc2))
    a.release()
    c.release()


def test_adjoint_after_skipping_forward():
    sc = _scene(0)
    grads = []
    for skip in (True, False):
        dev = _device(sc, skip=skip)
        g = torch.from_numpy(np.random.default_rng(5).normal(size=(len(sc.cams), sc.height, sc.width, 4))
                             .astype(np.float32)).cuda()
        dtf, dvol = dev.backward(g)
        grads.append((dtf.double().cpu(), dvol.double().cpu()))
        dev.release()
    (ta, va), (tb, vb) = grads
    # TF entries of opacity 0 still get a gradient (dalpha/da = sigma dt there)
    low = torch.from_numpy(sc.tf[:, 3] == 0.0)
    assert float(tb[low, 3].abs().max()) > 0.0
    # equal up to the order of the FP32 atomic sums
    for x, y in ((ta, tb), (va, vb)):
        assert float((x - y).norm()) <= 1e-5 * float(y.norm())
        assert float((x - y).abs().max()) <= 1e-5 * float(y.abs().max())


def test_refusals():
    sc = _scene(0)
    dev = _device(sc, skip=True)
    with pytest.raises(dpv.DPVError, match="UNSUPPORTED"):
        dev.set_frame(sc.width, sc.height, skip=True, iso=0.5)
    with pytest.raises(dpv.DPVError, match="UNSUPPORTED"):
        dev.set_frame(sc.width, sc.height, skip=True, staged=True)
    bricks = []
    for k in range(sc.part.num_ranks):
        stored, _, scale = dev.read_brick(k)
        bricks.append((sc.part.lo[k], sc.part.hi[k], stored.clone(), scale))
    dev.release()
    rgba = torch.zeros((sc.height, sc.width, 4), device="cuda")
    depth = torch.zeros((sc.height, sc.width), device="cuda")
    with pytest.raises(dpv.DPVError, match="UNSUPPORTED"):
        dpv.render_noalloc(sc.dims, bricks, "f32", torch.from_numpy(sc.tf).cuda(), sc.cams[0], sc.width, sc.height,
                           rgba, depth, flags=dpv.FRAME_SKIP)
