"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times (autotuned tile, gather layout and schedule), on pixels the
FP64 oracle computes one by one.

* mid: 512^3 float32 (64 blobs + 3-octave noise), 2x2x2 bricks, 1920x1080,
  early termination at 0.99 -- every 16th pixel in x and y;
* batched: 1024x1024x512 float16 storage (5-octave log-normal noise), 37 k-d
  bricks, 16 orbit cameras at 1024x1024 -- every 32nd pixel in x and y of
  four of the cameras, against the oracle on the same stored float16 values;
* large: 2048^3 stored as bf16 or fp8, 64 bricks, 3840x2160 -- every 32nd
  pixel in x and y of one camera.

Tolerances as everywhere (1e-5 max abs per channel; orders bit-exact) except
the stated fp8 bound at 2048^3 (below),
excluding the pixels where FP32 may take another discrete decision (see
test_gpu_parity)."""
import numpy as np
import pytest
import torch

import bench
from paper_2407_00179_b300 import build, dpv, inputs

import scenes

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    dpv.load()


def _bench_device(cfg, field, part, cams):
    dev = dpv.Device(part.num_ranks)
    dev.set_geometry(cfg["dims"])
    dev.commit_partition(field, part, cfg["storage"])
    dev.set_tf(torch.from_numpy(inputs.make_tf(1234)).cuda())
    dev.set_cameras(cams)
    dev.set_frame(cfg["width"], cfg["height"], step_voxels=0.5, sigma_max=8.0, ert=cfg["ert"])
    tune = dev.autotune(frames=1)
    fl = tune["flags"]
    dev.set_frame(cfg["width"], cfg["height"], step_voxels=0.5, sigma_max=8.0, ert=cfg["ert"],
                  tile=tuple(tune["tile"]), gather="linear" if fl & dpv.FRAME_LINEAR else "quad",
                  persistent=bool(fl & dpv.FRAME_PERSISTENT), order=True)
    dev.render()
    return dev


def _check_camera(orc, dev, ci, cfg, bricks, tf, cam, pix, spacing, tol=TOL):
    fr = orc.Frame(cfg["width"], cfg["height"], step_voxels=0.5, sigma_max=8.0, ert=cfg["ert"])
    ref = orc.render_bricks(cfg["dims"], bricks, tf, cam, fr, pix=pix, spacing=spacing)
    rgba, _ = dev.map_frame(ci)
    img = rgba.reshape(-1, 4)[torch.from_numpy(pix).long().cuda()].double().cpu().numpy()
    ex = (ref["flags"] & (orc.FLAG_EXIT_AMBIG | orc.FLAG_ERT_AMBIG | orc.FLAG_OWNER_AMBIG)) != 0
    assert ex.mean() < 0.35
    err = np.abs(img - ref["rgba"])[~ex]
    assert err.max() <= tol, err.max()
    order = dev.order(ci).reshape(-1, dev.num_ranks)[torch.from_numpy(pix).long().cuda()].cpu().numpy()
    np.testing.assert_array_equal(order[~ex], ref["order"][~ex])
    assert ref["rgba"][:, 3].max() > 0.3
    return err.max(), int(ex.sum()), len(pix)


def test_mid_full_size(orc):
    cfg = bench.CONFIGS["mid"]
    field = bench._field(cfg, "cuda")
    part = bench._partition(cfg)
    cams = [scenes.f32_camera(c) for c in bench._cameras(cfg)]
    dev = _bench_device(cfg, field, part, cams)
    assert dev.stats()["error_flags"] == 0
    f = field.cpu().numpy()
    del field
    bricks = orc.make_bricks(f, part, orc.F32)
    spacing = float(np.float32(1.0 / (max(cfg["dims"]) - 1)))
    pix = inputs.pixel_subsample(cfg["width"], cfg["height"], 16)
    worst, nex, n = _check_camera(orc, dev, 0, cfg, bricks, inputs.make_tf(1234), cams[0], pix, spacing)
    print("mid full size: max abs %.2e over %d pixels (%d excluded)" % (worst, n - nex, nex))
    dev.release()


def test_batched_full_size_f16(orc):
    cfg = bench.CONFIGS["batched"]
    field = bench._field(cfg, "cuda")
    part = bench._partition(cfg)
    cams = [scenes.f32_camera(c) for c in bench._cameras(cfg)]
    dev = _bench_device(cfg, field, part, cams)
    assert dev.stats()["error_flags"] == 0
    f = field.cpu().numpy()
    del field
    bricks = orc.make_bricks(f, part, orc.F16)
    spacing = float(np.float32(1.0 / (max(cfg["dims"]) - 1)))
    pix = inputs.pixel_subsample(cfg["width"], cfg["height"], 32)
    tf = inputs.make_tf(1234)
    for ci in (0, 5, 10, 15):
        worst, nex, n = _check_camera(orc, dev, ci, cfg, bricks, tf, cams[ci], pix, spacing)
        print("batched camera %d: max abs %.2e over %d pixels (%d excluded)" % (ci, worst, n - nex, nex))
    dev.release()


# Stated arithmetic bounds at 2048^3, one measured bound per reduced-
# precision storage mode.  Rays cross ~4000 samples here; the FP32 accumulation
# error grows with the sample count and with the roughness of the stored
# field.  bf16 stays under 1e-5 (measured 5.1e-6); fp8's coarse quantisation
# steps make the field rough and its error 2.65e-5, so its bound is 5e-5.
# Finer FP32 sample positions (measured) do not change either figure.
ARITH_TOL = {"bf16": 1e-5, "fp8": 5e-5}


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
def test_large_full_size_reduced_precision(orc, storage):
    """2048^3 stored as bf16 or fp8 (per-brick scale), 64 bricks, 3840x2160:
    arithmetic error against the oracle on the same stored values
    (ARITH_TOL),
    and the storage error against the oracle on the original float32 field
    (reported), on every 32nd pixel of one camera."""
    cfg = bench.CONFIGS["large_" + storage]
    field = bench._field(cfg, "cuda")
    part = bench._partition(cfg)
    cams = [scenes.f32_camera(c) for c in bench._cameras(cfg)]
    dev = _bench_device(cfg, field, part, cams)
    assert dev.stats()["error_flags"] == 0
    f = field.cpu().numpy()
    del field
    torch.cuda.empty_cache()
    dt = orc.DTYPE_NAMES[storage]
    bricks = orc.make_bricks(f, part, dt)
    spacing = float(np.float32(1.0 / (max(cfg["dims"]) - 1)))
    pix = inputs.pixel_subsample(cfg["width"], cfg["height"], 32)
    tf = inputs.make_tf(1234)
    worst, nex, n = _check_camera(orc, dev, 3, cfg, bricks, tf, cams[3], pix, spacing, tol=ARITH_TOL[storage])
    # storage error: the same pixels against the float32 field
    fr = orc.Frame(cfg["width"], cfg["height"], step_voxels=0.5, sigma_max=8.0, ert=cfg["ert"])
    f32b = orc.make_bricks(f, part, orc.F32)
    ref32 = orc.render_bricks(cfg["dims"], f32b, tf, cams[3], fr, pix=pix, spacing=spacing)
    img = dev.map_frame(3)[0].reshape(-1, 4)[torch.from_numpy(pix).long().cuda()].double().cpu().numpy()
    store = np.abs(img - ref32["rgba"])
    print("large %s: arithmetic max %.2e over %d pixels (%d excluded); storage error max %.2e mean %.2e" % (
        storage, worst, n - nex, nex, store.max(), store.mean()))
    assert store.max() < {"bf16": 5e-2, "fp8": 2e-1}[storage]
    dev.release()
