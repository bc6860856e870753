"""GPU visibility-ordered march with global early termination
(DPV_FRAME_ORDERED) against the FP64 oracle on the same stored values.

* 1e-5 max abs per RGBA channel on every pixel the oracle does not flag
  (the sample count at the volume's exit, a sample's brick at a brick face
  under per-brick fp8 scales, the accumulated opacity within 1e-4 of the
  threshold when the march stops), opaque (termination) and translucent
  scenes, regular and k-d partitions, a camera inside, f32/f16/fp8;
* evaluated samples: the GPU's count equals the oracle's up to the flagged
  pixels' rays;
* depth: t of the first sample of the first brick segment that adds
  opacity, 1e-5 relative, excluding segments whose FP64 opacity is below
  1e-6 (FP32 may not resolve them);
* without termination it equals the sort-last frame within 1e-5; with it
  on an opaque scene it evaluates fewer samples than per-fragment
  termination; launch layouts agree bit for bit; the adjoint refuses it.
"""
import numpy as np
import pytest
import torch

from paper_2407_00179_b300 import build, dpv, inputs

import scenes

pytestmark = pytest.mark.gpu

TOL = 1e-5

CASES = [
    dict(dims=(48, 40, 44), splits=(2, 2, 2), width=96, height=80, sigma_max=60.0, ert=0.95),
    dict(dims=(50, 42, 36), kd=9, width=67, height=45, tile=(8, 4), sigma_max=80.0, ert=0.99),
    dict(dims=(50, 42, 36), kd=5, width=61, height=47, tile=(32, 8), inside=True, sigma_max=60.0, ert=0.9),
    dict(dims=(40, 36, 32), splits=(2, 2, 2), width=48, height=40, storage="f16", sigma_max=8.0, ert=0.99),
    dict(dims=(40, 36, 32), splits=(2, 1, 2), width=52, height=44, storage="fp8", sigma_max=50.0, ert=0.95),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    dpv.load()


def _scene(i):
    c = dict(CASES[i])
    inside = c.pop("inside", False)
    dims = c.pop("dims")
    cams = inputs.random_cameras(dims, 2, seed=60 + i, inside=inside)
    return scenes.make(dims, cams=cams, nblobs=10, seed=i, **c)


def _device(sc, ordered=True, gather="auto"):
    dev = scenes.gpu_device(sc, order=False)
    dev.set_frame(sc.width, sc.height, step_voxels=sc.step, sigma_max=sc.sigma_max, ert=sc.ert, tile=sc.tile,
                  gather=gather, ordered=ordered)
    dev.render()
    return dev


@pytest.mark.parametrize("i", range(len(CASES)))
def test_ordered_matches_fp64_oracle(orc, i):
    sc = _scene(i)
    dev = _device(sc)
    st = dev.stats()
    assert st["error_flags"] == 0
    bricks = scenes.oracle_bricks(orc, sc)
    fr = scenes.oracle_frame(orc, sc)
    n_ref = n_flag = 0
    stopped = 0
    for ci, cam in enumerate(sc.cams):
        ref = orc.render_ordered(sc.dims, sc.tf, cam, fr, bricks=bricks, spacing=sc.spacing)
        # every sample of the ray (the count depends on the geometry only)
        full = orc.render_full(sc.field, sc.tf, cam, orc.Frame(sc.width, sc.height, step_voxels=sc.step,
                                                               sigma_max=sc.sigma_max), spacing=sc.spacing)
        rgba, depth = dev.map_frame(ci)
        rgba = rgba.reshape(-1, 4).double().cpu().numpy()
        depth = depth.reshape(-1).double().cpu().numpy()
        amb = scenes.FLAG["exit"] | scenes.FLAG["ert"] | (scenes.FLAG["owner"] if sc.storage == "fp8" else 0)
        ok = (ref["flags"] & amb) == 0
        assert ok.mean() > 0.9
        err = np.abs(rgba - ref["rgba"])[ok]
        assert err.max() <= TOL, err.max()
        fin = ok & np.isfinite(ref["depth"]) & (ref["depth_alpha"] > 1e-6)
        np.testing.assert_array_equal(np.isinf(depth[ok & (ref["depth_alpha"] == 0)]),
                                      np.isinf(ref["depth"][ok & (ref["depth_alpha"] == 0)]))
        if fin.any():
            assert np.abs(depth[fin] - ref["depth"][fin]).max() <= 1e-5 * np.abs(ref["depth"][fin]).max()
        n_ref += int(ref["nsamples"].sum())
        n_flag += int(full["nsamples"][~ok].sum())
        stopped += int((ref["nsamples"] < full["nsamples"]).sum())
        assert ref["rgba"][:, 3].max() > 0.3
    assert abs(st["samples_forward"] - n_ref) <= n_flag
    if sc.sigma_max > 10:
        assert stopped > 50                     # termination actually happens
    dev.release()


def test_without_termination_equals_sort_last():
    sc = _scene(3)
    sc.ert = 0.0
    a = _device(sc, ordered=True)
    b = _device(sc, ordered=False)
    for c in range(len(sc.cams)):
        ra, da = a.map_frame(c)
        rb, db = b.map_frame(c)
        assert float((ra - rb).abs().max()) <= TOL
    assert a.stats()["samples_forward"] == b.stats()["samples_forward"]
    a.release()
    b.release()


def test_fewer_samples_than_per_fragment_termination():
    sc = _scene(0)
    a = _device(sc, ordered=True)
    b = _device(sc, ordered=False)
    na, nb = a.stats()["samples_forward"], b.stats()["samples_forward"]
    print("ordered %d samples, sort-last %d (%.2f)" % (na, nb, na / nb))
    assert na < 0.9 * nb
    a.release()
    b.release()


def test_ordered_layouts_agree_and_refusals():
    sc = _scene(1)
    frames = []
    for gather in ("cell", "quad", "linear"):
        dev = _device(sc, gather=gather)
        frames.append([torch.cat([t.reshape(-1) for t in dev.map_frame(c)]).clone() for c in range(len(sc.cams))])
        if gather == "cell":
            with pytest.raises(dpv.DPVError, match="UNSUPPORTED"):
                dev.backward(torch.zeros((len(sc.cams), sc.height, sc.width, 4), device="cuda"))
            with pytest.raises(dpv.DPVError, match="UNSUPPORTED"):
                dev.set_frame(sc.width, sc.height, ordered=True, iso=0.5)
        dev.release()
    for other in frames[1:]:
        for a, b in zip(frames[0], other):
            assert torch.equal(a, b)


def _ordered_outputs(sc, gather, skip, order, persistent):
    dev = scenes.gpu_device(sc, order=False)
    dev.set_frame(sc.width, sc.height, step_voxels=sc.step, sigma_max=sc.sigma_max, ert=sc.ert, tile=sc.tile,
                  gather=gather, ordered=True, order=order, skip=skip, persistent=persistent)
    dev.render()
    assert dev.stats()["error_flags"] == 0
    frames = [torch.cat([t.reshape(-1) for t in dev.map_frame(c)]).clone() for c in range(len(sc.cams))]
    orders = [dev.order(c).clone() for c in range(len(sc.cams))] if order else []
    n = dev.stats()["samples_forward"]
    dev.release()
    return frames, orders, n


@pytest.mark.parametrize("i", range(len(CASES)))
def test_persistent_form_is_bit_identical(i):
    """The persistent form (DPV_FRAME_PERSISTENT: warps pull 32 pixels at a
    time) writes the per-tile form's colour, depth and order map bit for bit
    and evaluates the same samples: every layout, with and without
    empty-space skipping, with and without the order map (a terminated ray
    still lists the segments behind it)."""
    sc = _scene(i)
    for gather in ("cell", "quad", "linear"):
        for skip, order in ((False, False), (True, False), (False, True)):
            fa, oa, na = _ordered_outputs(sc, gather, skip, order, persistent=False)
            fb, ob, nb = _ordered_outputs(sc, gather, skip, order, persistent=True)
            assert na == nb, (gather, skip, order, na, nb)
            for a, b in zip(fa, fb):
                assert torch.equal(a, b), (gather, skip, order)
            for a, b in zip(oa, ob):
                assert torch.equal(a, b), (gather, skip, order)


def test_long_work_lists_scan_the_list(orc):
    """Tile lists longer than the per-ray entry cache (16 items) take the
    scanning selection: one 16x16 tile that sees the whole of a 40-brick k-d
    partition (a wide field of view), both launch forms and every layout bit
    for bit, and the frame against the oracle."""
    dims = (64, 60, 56)
    c = inputs.camera_from_direction(dims, (1.0, 0.7, 0.5))
    cam = inputs.Camera(c.eye, c.center, c.up, 100.0)
    sc = scenes.make(dims, kd=40, cams=[cam], nblobs=10, seed=3, width=16, height=16, tile=(16, 16),
                     sigma_max=60.0, ert=0.95)
    dev = _device(sc)
    st = dev.stats()
    assert st["work_items"] > 16                        # the one tile's list
    dev.release()
    ref_frames = None
    for gather in ("cell", "quad", "linear"):
        for persistent in (False, True):
            f, _, n = _ordered_outputs(sc, gather, False, False, persistent=persistent)
            if ref_frames is None:
                ref_frames, ref_n = f, n
            assert n == ref_n
            for a, b in zip(f, ref_frames):
                assert torch.equal(a, b), (gather, persistent)
    ref = orc.render_ordered(sc.dims, sc.tf, sc.cams[0], scenes.oracle_frame(orc, sc),
                             bricks=scenes.oracle_bricks(orc, sc), spacing=sc.spacing)
    rgba = ref_frames[0][:sc.width * sc.height * 4].reshape(-1, 4).double().cpu().numpy()
    ok = (ref["flags"] & (scenes.FLAG["exit"] | scenes.FLAG["ert"])) == 0
    assert ok.mean() > 0.8 and ref["rgba"][:, 3].max() > 0.3
    assert np.abs(rgba - ref["rgba"])[ok].max() <= TOL
