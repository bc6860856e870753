"""GPU iso-surface fragments (DPV_FRAME_ISO) against the FP64 oracle on the
same stored values.

* hit or no hit, and the nearest key (the smallest per-brick fragment key),
  bit-exact on every pixel the oracle does not flag (a sample within 5e-5
  of the level up to the hit, a surface point within 1e-4 of a cell face,
  the sample count, or under fp8's per-brick scales a sample near a brick
  face, may be decided otherwise in FP32);
* depth: |gpu - ref| <= dt 8e-6 / |s_h - s_{h-1}| + 2e-6 (1 + depth): the
  interpolated fraction moves by the samples' FP32 error over the pair's
  difference (measured worst: 0.15 of this bound);
* colour: 2e-6 max abs per channel on hits whose pair differs by at least
  1e-2 (measured worst 3e-7);
* the three gather layouts give identical frames; the adjoint and the
  staged form refuse iso frames.
"""
import numpy as np
import pytest
import torch

from paper_2407_00179_b300 import build, dpv, inputs

import scenes

pytestmark = pytest.mark.gpu

CASES = [
    dict(dims=(48, 40, 44), splits=(2, 2, 2), width=96, height=80, iso=0.3),
    dict(dims=(50, 42, 36), kd=9, width=67, height=45, tile=(8, 4), iso=0.55),
    dict(dims=(50, 42, 36), kd=5, width=61, height=47, tile=(32, 8), inside=True, iso=0.45),
    dict(dims=(40, 36, 32), splits=(2, 2, 2), width=48, height=40, storage="f16", iso=0.35),
    dict(dims=(40, 36, 32), splits=(2, 1, 2), width=52, height=44, storage="fp8", iso=0.4),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    dpv.load()


def _scene(i):
    c = dict(CASES[i])
    inside = c.pop("inside", False)
    dims = c.pop("dims")
    iso = c.pop("iso")
    cams = inputs.random_cameras(dims, 2, seed=40 + i, inside=inside)
    return scenes.make(dims, cams=cams, nblobs=10, seed=i, **c), iso


def _device(sc, iso, gather="auto"):
    dev = scenes.gpu_device(sc, order=False)
    dev.set_frame(sc.width, sc.height, step_voxels=sc.step, sigma_max=sc.sigma_max, tile=sc.tile, gather=gather,
                  iso=iso)
    dev.render()
    return dev


@pytest.mark.parametrize("i", range(len(CASES)))
def test_iso_matches_fp64_oracle(orc, i):
    sc, iso = _scene(i)
    dev = _device(sc, iso)
    assert dev.stats()["error_flags"] == 0
    bricks = scenes.oracle_bricks(orc, sc)
    fr = scenes.oracle_frame(orc, sc)
    dt = sc.step * sc.spacing
    nhit = ncol = 0
    worst_d = worst_c = 0.0
    for ci, cam in enumerate(sc.cams):
        ref = orc.render_iso(sc.dims, sc.tf, cam, fr, iso, bricks=bricks, spacing=sc.spacing)
        rgba, depth = dev.map_frame(ci)
        rgba = rgba.reshape(-1, 4).double().cpu().numpy()
        depth = depth.reshape(-1).double().cpu().numpy()
        keys = np.stack([dev.read_fragments(ci, k)[1].reshape(-1).cpu().numpy() for k in range(sc.part.num_ranks)], 1)
        gkey = keys.astype(np.int64).min(axis=1)
        gkey[gkey == 2 ** 31 - 1] = -1
        # ambiguous pixels; ownership only matters where per-brick scales
        # differ (fp8): ghost copies are otherwise equal
        amb = orc.FLAG_ISO_AMBIG | orc.FLAG_EXIT_AMBIG | (orc.FLAG_OWNER_AMBIG if sc.storage == "fp8" else 0)
        ok = (ref["flags"] & amb) == 0
        assert ok.mean() > 0.9
        # hit / no hit and the nearest key
        np.testing.assert_array_equal(gkey[ok], ref["key"][ok])
        np.testing.assert_array_equal(rgba[ok, 3], ref["rgba"][ok, 3])
        hit = ok & (ref["key"] >= 0)
        miss = ok & (ref["key"] < 0)
        assert np.all(np.isinf(depth[miss])) and np.all(rgba[miss] == 0.0)
        # depth, bounded by the pair's conditioning
        tol = dt * 8e-6 / np.maximum(ref["dsdt"][hit], 1e-30) + 2e-6 * (1.0 + np.abs(ref["depth"][hit]))
        err = np.abs(depth[hit] - ref["depth"][hit])
        assert np.all(err <= tol), (err.max(), tol[np.argmax(err / tol)])
        worst_d = max(worst_d, float((err / tol).max()) if len(err) else 0.0)
        # colour where the crossing is well conditioned
        good = hit & (ref["dsdt"] >= 1e-2)
        cerr = np.abs(rgba[good, :3] - ref["rgba"][good, :3])
        if cerr.size:
            assert cerr.max() <= 2e-6, cerr.max()
            worst_c = max(worst_c, float(cerr.max()))
        nhit += int(hit.sum())
        ncol += int(good.sum())
    print("iso case %d: %d hits, %d colour-checked, depth err / bound max %.2e, colour max %.2e"
          % (i, nhit, ncol, worst_d, worst_c))
    assert nhit > 50 and ncol > 20
    dev.release()


def test_iso_gather_layouts_agree():
    sc, iso = _scene(1)
    frames = []
    for gather in ("cell", "quad", "linear"):
        dev = _device(sc, iso, gather)
        frames.append([torch.cat([t.reshape(-1) for t in dev.map_frame(c)]).clone() for c in range(len(sc.cams))])
        dev.release()
    for a, b in zip(frames[0], frames[1]):
        assert torch.equal(a, b)
    for a, b in zip(frames[0], frames[2]):
        assert torch.equal(a, b)


def test_iso_refusals():
    sc, iso = _scene(0)
    dev = _device(sc, iso)
    with pytest.raises(dpv.DPVError, match="UNSUPPORTED"):
        dev.backward(torch.zeros((len(sc.cams), sc.height, sc.width, 4), device="cuda"))
    with pytest.raises(dpv.DPVError, match="UNSUPPORTED"):
        dev.set_frame(sc.width, sc.height, staged=True, iso=iso)
    dev.release()
