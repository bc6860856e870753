"""Batched launch forms against the plain one: the persistent brick-major
ray-march, CUDA-graph replay and the autotuner's choice must all give frames
and fragments bit-identical to one-CTA-per-item launches (each work item is
computed by the same code whatever the order), and adjoints equal up to
atomic summation order."""
import numpy as np
import pytest
import torch

from paper_2407_00179_b300 import build, dpv, inputs

import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    dpv.load()


def _scene(i):
    if i == 0:
        dims = (48, 40, 44)
        return scenes.make(dims, kd=11, cams=inputs.orbit_cameras(dims, 6, seed=3), width=80, height=64)
    if i == 1:
        dims = (50, 42, 36)
        return scenes.make(dims, splits=(2, 2, 2), cams=inputs.random_cameras(dims, 3, seed=8, inside=True),
                           width=67, height=45, storage="f16", ert=0.99)
    dims = (40, 36, 32)
    return scenes.make(dims, splits=(3, 1, 2), cams=inputs.sphere_cameras(dims, 4, seed=2), width=48, height=40,
                       storage="fp8", tile=(8, 4))


def _device(sc, **kw):
    dev = scenes.gpu_device(sc, order=True)
    dev.set_frame(sc.width, sc.height, step_voxels=sc.step, sigma_max=sc.sigma_max, ert=sc.ert, tile=sc.tile,
                  order=True, **kw)
    dev.render()
    return dev


def _same_frames(a, b, sc):
    for c in range(len(sc.cams)):
        assert torch.equal(a.map_frame(c)[0], b.map_frame(c)[0])
        assert torch.equal(a.map_frame(c)[1], b.map_frame(c)[1])
        assert torch.equal(a.order(c), b.order(c))


@pytest.mark.parametrize("i", range(3))
def test_persistent_brick_major_equals_per_item(i):
    sc = _scene(i)
    a = _device(sc)
    b = _device(sc, persistent=True)
    _same_frames(a, b, sc)
    for k in range(sc.part.num_ranks):
        assert torch.equal(a.read_fragments(0, k)[0], b.read_fragments(0, k)[0])
    assert a.stats()["samples_forward"] == b.stats()["samples_forward"]
    g = torch.from_numpy(inputs.rng(i, inputs.STREAM_GRAD).normal(
        size=(len(sc.cams), sc.height, sc.width, 4)).astype(np.float32)).cuda()
    ta, va = a.backward(g)
    tb, vb = b.backward(g)
    assert a.stats()["samples_backward"] == b.stats()["samples_backward"]
    assert torch.allclose(ta, tb, rtol=1e-4, atol=1e-7 * float(ta.abs().max()))
    assert torch.allclose(va, vb, rtol=1e-4, atol=1e-6 * float(va.abs().max()))
    a.release()
    b.release()


@pytest.mark.parametrize("i", range(3))
def test_graph_replay_equals_direct_and_follows_tf_updates(i):
    sc = _scene(i)
    a = _device(sc, persistent=True)
    b = _device(sc, persistent=True, graph=True)
    b.render()                                   # a replay of the captured graph
    _same_frames(a, b, sc)
    tf2 = torch.from_numpy(inputs.perturb_tf(sc.tf, seed=i)).cuda()
    a.set_tf(tf2)
    b.set_tf(tf2)
    a.render()
    b.render()
    _same_frames(a, b, sc)
    assert b.stats()["samples_forward"] == a.stats()["samples_forward"]
    assert b.stats()["graph_launches"] >= 2 and a.stats()["graph_launches"] == 0
    a.release()
    b.release()


def test_autotune_choice_renders_the_same_frame(tmp_path):
    sc = _scene(0)
    ref = _device(sc)
    dev = _device(sc)
    res = dev.autotune(frames=2, cache=str(tmp_path / "tune.json"), key="scene0")
    # 4 tiles x {cell, quad, linear} x {per-item, persistent}: the cell
    # layout of this small scene always fits
    assert res["candidates"] == 24 and res["ms"] > 0 and not res["cached"]
    assert res["tile"] in ([16, 16], [32, 8], [8, 32], [64, 4])
    assert dpv.gather_of(res["flags"]) in ("cell", "quad", "linear")
    _same_frames(ref, dev, sc)
    # a second device picks the stored choice without timing
    dev2 = _device(sc)
    res2 = dev2.autotune(cache=str(tmp_path / "tune.json"), key="scene0")
    assert res2["cached"] and res2["tile"] == res["tile"] and res2["flags"] == res["flags"]
    dev2.render()
    _same_frames(ref, dev2, sc)
    for d in (ref, dev, dev2):
        d.release()


def test_async_frame_copies_in_flight():
    """dpvCopyFrameAsync: frames of successive renders (different TFs)
    copied to pinned host memory while the next render runs, more copies in
    flight than staging slots, single cameras and all cameras at once: each
    destination holds the frame of the render before its copy."""
    sc = _scene(0)
    dev = _device(sc)
    ncam, H, W = len(sc.cams), sc.height, sc.width
    tfs = [inputs.make_tf(1234), inputs.make_tf(77), inputs.make_tf(5), inputs.make_tf(9)]
    want, outs = [], []
    for k, tf in enumerate(tfs):
        dev.set_tf(torch.from_numpy(tf).cuda())
        dev.render()
        if k % 2 == 0:
            rgba = torch.empty((ncam, H, W, 4), dtype=torch.float32).pin_memory()
            depth = torch.empty((ncam, H, W), dtype=torch.float32).pin_memory()
            dev.copy_frame_async(-1, rgba, depth)
            outs.append((rgba, depth))
            want.append([t.clone() for c in range(ncam) for t in dev.map_frame(c)])
        else:
            rgba = torch.empty((H, W, 4), dtype=torch.float32).pin_memory()
            dev.copy_frame_async(ncam - 1, rgba, None)
            outs.append((rgba, None))
            want.append([dev.map_frame(ncam - 1)[0].clone()])
    dev.copy_wait()
    torch.cuda.synchronize()
    for k, ((rgba, depth), w) in enumerate(zip(outs, want)):
        if depth is not None:
            for c in range(ncam):
                assert torch.equal(rgba[c], w[2 * c].cpu())
                assert torch.equal(depth[c], w[2 * c + 1].cpu())
        else:
            assert torch.equal(rgba, w[0].cpu())
    # successive frames differ, so a stale slot would show
    assert not torch.equal(outs[0][0][ncam - 1], outs[1][0])
    with pytest.raises(dpv.DPVError, match="INVALID_ARG"):
        dev.copy_frame_async(ncam, outs[1][0], None)
    dev.release()


@pytest.mark.parametrize("mode", ["skip", "deep", "shadow"])
def test_graph_replay_of_the_extended_modes(mode):
    """Skipping, deep fragments and shadows replayed from a CUDA graph give
    the direct launches' frames bit for bit, also after a TF update (the
    skipping classification and the shadows read the new table)."""
    sc = _scene(1)
    kw = {"skip": dict(skip=True), "deep": dict(deep=True), "shadow": dict(shadow=True)}[mode]
    tfs = [inputs.make_tf(1234, transparent_below=0.3), inputs.make_tf(55, transparent_below=0.2)]
    frames = []
    for graph in (False, True):
        dev = scenes.gpu_device(sc, order=False)
        if mode == "shadow":
            dev.set_light((0.3, 0.8, 0.5), 1.0, 0.25)
        dev.set_frame(sc.width, sc.height, step_voxels=sc.step, sigma_max=sc.sigma_max, ert=sc.ert, tile=sc.tile,
                      graph=graph, **kw)
        out = []
        for tf in tfs:
            dev.set_tf(torch.from_numpy(tf).cuda())
            for _ in range(2):
                dev.render()
            out.append([t.clone() for c in range(len(sc.cams)) for t in dev.map_frame(c)])
        if graph:
            assert dev.stats()["graph_launches"] > 0
        frames.append(out)
        dev.release()
    for a, b in zip(frames[0], frames[1]):
        for x, y in zip(a, b):
            assert torch.equal(x, y)
    assert not torch.equal(frames[0][0][0], frames[0][1][0])      # the TF update changed the frame
