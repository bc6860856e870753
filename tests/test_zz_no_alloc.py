"""The allocation-free render entry point, dpvRenderNoAlloc.

Some callers cannot let a library allocate device memory: applications whose
GPU memory is owned by their own pool or by a framework's caching allocator,
and render loops that cannot afford the device-wide synchronisation of
cudaMalloc/cudaFree.  dpvRenderNoAlloc renders one camera from caller-owned
inputs into caller-owned outputs, keeping its intermediates in one fixed
device array inside the library.  These tests check, through the C ABI, that
it gives the same frame as the regular entry point (dpvRenderFrame) within
the parity tolerance for every storage format, on calls made back to back
(the shared array keeps the previous call's contents); that its frame
matches the FP64 oracle directly; that the largest documented frame fits
and later calls change no device memory figure; and that it refuses frames
too large for the array, misaligned tables, degenerate cameras and flags
that need device state.  This file is collected last so that a failure here
leaves every other test already run.
"""
import numpy as np
import pytest
import torch

from paper_2407_00179_b300 import build, dpv, inputs

import scenes

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    dpv.load()


def _reference(sc):
    """Frame of the regular entry point and the committed bricks, read back
    as caller-owned device tensors for the allocation-free call."""
    dev = scenes.gpu_device(sc, order=False)
    dev.render()
    rgba, depth = dev.map_frame(0)
    ref = (rgba.clone(), depth.clone())
    bricks = []
    for k in range(sc.part.num_ranks):
        stored, _, scale = dev.read_brick(k)
        bricks.append((sc.part.lo[k], sc.part.hi[k], stored.clone(), scale))
    dev.release()
    return ref, bricks


def _noalloc(sc, bricks, tf):
    rgba = torch.full((sc.height, sc.width, 4), float("nan"), device="cuda")
    depth = torch.full((sc.height, sc.width), float("nan"), device="cuda")
    dpv.render_noalloc(sc.dims, bricks, sc.storage, tf, sc.cams[0], sc.width, sc.height, rgba, depth,
                       step_voxels=sc.step, sigma_max=sc.sigma_max, ert=sc.ert, tile=sc.tile, spacing=sc.spacing)
    torch.cuda.synchronize()
    return rgba, depth


def _same(a, b):
    (ra, da), (rb, db) = a, b
    assert torch.isfinite(ra).all()
    assert float((ra - rb).abs().max()) <= TOL
    fin = torch.isfinite(db)
    assert torch.equal(torch.isfinite(da), fin)
    assert float((da[fin] - db[fin]).abs().max()) <= TOL * float(db[fin].abs().max())


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16", "fp8"])
def test_matches_render_frame_on_consecutive_calls(storage):
    sc = scenes.make((48, 40, 44), kd=7, width=96, height=80, storage=storage, ert=0.99)
    ref, bricks = _reference(sc)
    if storage == "fp8":
        assert all(b[3] != 1.0 for b in bricks)        # the per-brick scales are in play
    tf = torch.from_numpy(sc.tf).cuda()
    for _ in range(2):
        _same(_noalloc(sc, bricks, tf), ref)


@pytest.mark.parametrize("storage", ["f32", "fp8"])
def test_matches_the_oracle(orc, storage):
    """The allocation-free frame against the FP64 oracle on the same stored
    values, directly (1e-5 per channel on the pixels the oracle does not
    flag), for a k-d partition and for a single rank (K = 1)."""
    for sc in (scenes.make((48, 40, 44), kd=7, width=96, height=80, storage=storage),
               scenes.make((40, 36, 30), splits=(1, 1, 1), width=64, height=48, storage=storage)):
        _, bricks = _reference(sc)
        rgba, _ = _noalloc(sc, bricks, torch.from_numpy(sc.tf).cuda())
        ref = scenes.o_bricks(orc, sc, sc.cams[0])
        ok = (ref["flags"] & (scenes.FLAG["exit"] | scenes.FLAG["owner"])) == 0
        assert ok.mean() > 0.95
        err = np.abs(rgba.double().cpu().numpy().reshape(-1, 4) - ref["rgba"])[ok]
        assert err.max() <= TOL, err.max()
        assert ref["rgba"][:, 3].max() > 0.3


def test_largest_documented_frame_allocates_nothing():
    """512 x 512 with 8 ranks fits the fixed array.  Once a first call has
    loaded the library's kernels, later calls leave the device's free memory
    and the caching allocator's count unchanged."""
    sc = scenes.make((48, 40, 44), splits=(2, 2, 2), width=512, height=512)
    ref, bricks = _reference(sc)
    tf = torch.from_numpy(sc.tf).cuda()
    rgba = torch.empty((sc.height, sc.width, 4), device="cuda")
    depth = torch.empty((sc.height, sc.width), device="cuda")

    def call():
        dpv.render_noalloc(sc.dims, bricks, sc.storage, tf, sc.cams[0], sc.width, sc.height, rgba, depth,
                           spacing=sc.spacing)
        torch.cuda.synchronize()

    call()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for _ in range(2):
        call()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    _same((rgba, depth), ref)


def test_refusals():
    """A transfer function that is not 16-byte aligned, a camera whose eye
    is its center, and flags that need device state are refused."""
    sc = scenes.make((36, 30, 28), splits=(2, 1, 1), width=32, height=32)
    _, bricks = _reference(sc)
    rgba = torch.empty((32, 32, 4), device="cuda")
    depth = torch.empty((32, 32), device="cuda")
    big = torch.from_numpy(np.concatenate([sc.tf.reshape(-1), np.zeros(4, np.float32)])).cuda()
    shifted = big[1:1 + sc.tf.size].view(sc.tf.shape)           # 4 bytes off a 16-byte boundary
    with pytest.raises(dpv.DPVError) as e:
        dpv.render_noalloc(sc.dims, bricks, "f32", shifted, sc.cams[0], 32, 32, rgba, depth, spacing=sc.spacing)
    assert e.value.status == 1 and "aligned" in str(e.value)
    c = sc.cams[0]
    bad = inputs.Camera(c.eye, c.eye, c.up, c.fovy_deg)
    tf = torch.from_numpy(sc.tf).cuda()
    with pytest.raises(dpv.DPVError) as e:
        dpv.render_noalloc(sc.dims, bricks, "f32", tf, bad, 32, 32, rgba, depth, spacing=sc.spacing)
    assert e.value.status == 1 and "eye == center" in str(e.value)
    for flag in (dpv.FRAME_ORDER, dpv.FRAME_DEEP, dpv.FRAME_SHADOW, dpv.FRAME_ISO):
        with pytest.raises(dpv.DPVError) as e:
            dpv.render_noalloc(sc.dims, bricks, "f32", tf, c, 32, 32, rgba, depth, spacing=sc.spacing, flags=flag)
        assert e.value.status == 6


def test_alternating_scenes_do_not_leak_state():
    a = scenes.make((48, 40, 44), splits=(2, 2, 2), width=96, height=80)
    cams = inputs.random_cameras((36, 30, 28), 1, seed=5, inside=True)
    b = scenes.make((36, 30, 28), splits=(3, 1, 2), cams=cams, width=72, height=56, tile=(8, 4))
    ref_a, bricks_a = _reference(a)
    ref_b, bricks_b = _reference(b)
    tf = torch.from_numpy(a.tf).cuda()
    _same(_noalloc(a, bricks_a, tf), ref_a)
    _same(_noalloc(b, bricks_b, tf), ref_b)
    _same(_noalloc(a, bricks_a, tf), ref_a)


def test_rejects_frames_beyond_the_scratch_limit():
    sc = scenes.make((48, 40, 44), splits=(2, 2, 2), width=4096, height=4096)
    _, bricks = _reference(scenes.make((48, 40, 44), splits=(2, 2, 2), width=16, height=16))
    tf = torch.from_numpy(sc.tf).cuda()
    rgba = torch.empty((16, 16, 4), device="cuda")
    depth = torch.empty((16, 16), device="cuda")
    with pytest.raises(dpv.DPVError) as e:
        dpv.render_noalloc(sc.dims, bricks, "f32", tf, sc.cams[0], 4096, 4096, rgba, depth, spacing=sc.spacing)
    assert e.value.status == 1 and "scratch" in str(e.value)
