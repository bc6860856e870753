"""The shared-memory staged ray-march (DPV_FRAME_STAGED) against the default
march that gathers through L1: with float32 bricks both evaluate exactly the same
arithmetic on the same corner values, so fragments, frames and sample counts
must be bit-identical; the adjoints differ only in atomic summation order.
Also covers the fallback for slabs whose box does not fit in shared memory
(forced with a tiny DPV_BOX_CAP in a subprocess)."""
import os
import subprocess
import sys

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


SCENES = [
    dict(dims=(48, 40, 44), splits=(2, 2, 2), width=96, height=80),
    dict(dims=(50, 42, 36), kd=9, width=67, height=45, tile=(8, 4)),
    dict(dims=(50, 42, 36), kd=5, width=61, height=47, tile=(32, 8), inside=True),
    dict(dims=(64, 64, 64), splits=(2, 1, 1), width=256, height=256, ert=0.99, sigma_max=40.0),
    dict(dims=(40, 36, 32), splits=(2, 2, 2), width=48, height=40, storage="f16"),
]


def _scene(i):
    c = dict(SCENES[i])
    inside = c.pop("inside", False)
    dims = c.pop("dims")
    cams = inputs.random_cameras(dims, 2, seed=10 + i, inside=inside)
    return scenes.make(dims, cams=cams, **c)


def _render(sc, staged):
    sc.staged = staged
    dev = scenes.gpu_device(sc, order=True)
    dev.render()
    return dev


@pytest.mark.parametrize("i", range(len(SCENES)))
def test_staged_equals_unstaged_bitwise(i):
    sc = _scene(i)
    a = _render(sc, True)
    b = _render(sc, False)
    for c in range(len(sc.cams)):
        fa, fb = a.map_frame(c), b.map_frame(c)
        assert torch.equal(fa[0], fb[0])
        assert torch.equal(fa[1], fb[1])
        for k in range(sc.part.num_ranks):
            ra, ka = a.read_fragments(c, k)
            rb, kb = b.read_fragments(c, k)
            assert torch.equal(ka, kb)
            assert torch.equal(ra, rb)
    sa, sb = a.stats(), b.stats()
    assert sa["samples_forward"] == sb["samples_forward"]
    assert sa["error_flags"] == 0 and sb["error_flags"] == 0
    a.release()
    b.release()


@pytest.mark.parametrize("i", [0, 1, 3])
def test_staged_adjoint_matches_unstaged(i):
    sc = _scene(i)
    g = torch.from_numpy(inputs.rng(i, inputs.STREAM_GRAD).normal(
        size=(len(sc.cams), sc.height, sc.width, 4)).astype(np.float32)).cuda()
    a = _render(sc, True)
    b = _render(sc, False)
    ta, va = a.backward(g)
    tb, vb = b.backward(g)
    assert a.stats()["samples_backward"] == b.stats()["samples_backward"]
    assert a.stats()["error_flags"] == 0
    # the staged adjoint sums TF gradients in FP64 shared memory, the default
    # in FP32 per-lane-group copies: equal up to summation rounding
    assert torch.allclose(ta, tb, rtol=1e-4, atol=1e-7 * float(tb.abs().max()))
    assert torch.allclose(va, vb, rtol=1e-4, atol=1e-6 * float(vb.abs().max()))
    a.release()
    b.release()


def test_oversized_slabs_fall_back_to_global_memory(tmp_path):
    """With a 40-float box budget no slab fits: every slab takes the global
    path, and the results must not change."""
    code = r'''
import sys, torch, numpy as np
sys.path.insert(0, "tests")
import scenes
from paper_2407_00179_b300 import inputs
sc = scenes.make((48, 40, 44), kd=7, width=64, height=48)
sc.staged = True
dev = scenes.gpu_device(sc, order=False)
dev.render()
img = dev.map_frame(0)[0].cpu().numpy()
g = torch.ones((1, 48, 64, 4), device="cuda")
tf, vol = dev.backward(g)
np.savez(sys.argv[1], img=img, tf=tf.cpu().numpy(), vol=vol.cpu().numpy(), err=dev.stats()["error_flags"])
'''
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = {}
    for cap in ("40", "6144"):
        path = str(tmp_path / ("boxcap_%s.npz" % cap))
        env = dict(os.environ, DPV_BOX_CAP=cap)
        subprocess.check_call([sys.executable, "-c", code, path], cwd=root, env=env)
        out[cap] = np.load(path)
    a, b = out["40"], out["6144"]
    assert int(a["err"]) == 0 and int(b["err"]) == 0
    np.testing.assert_array_equal(a["img"], b["img"])
    np.testing.assert_allclose(a["tf"], b["tf"], rtol=1e-4, atol=1e-7 * np.abs(b["tf"]).max())
    np.testing.assert_allclose(a["vol"], b["vol"], rtol=1e-4, atol=1e-6 * np.abs(b["vol"]).max())


@pytest.mark.parametrize("other", ["linear", "cell"])
@pytest.mark.parametrize("i", range(len(SCENES)))
def test_gather_layouts_agree(i, other):
    """The default gather layout (2x2 corners per vector), the cell layout
    (eight corners per vector) and the eight-load path read the same stored
    values: identical frames and fragments, and the adjoint differs only in
    atomic summation order."""
    sc = _scene(i)
    sc.staged = False
    devs = []
    for gather in ("quad", other):
        dev = scenes.gpu_device(sc, order=False)
        dev.set_frame(sc.width, sc.height, step_voxels=sc.step, sigma_max=sc.sigma_max, ert=sc.ert, tile=sc.tile,
                      gather=gather)
        dev.render()
        devs.append(dev)
    a, b = devs
    for c in range(len(sc.cams)):
        assert torch.equal(a.map_frame(c)[0], b.map_frame(c)[0])
        for k in range(sc.part.num_ranks):
            assert torch.equal(a.read_fragments(c, k)[0], b.read_fragments(c, k)[0])
    assert a.stats()["samples_forward"] == b.stats()["samples_forward"]
    g = torch.from_numpy(inputs.rng(i, inputs.STREAM_GRAD).normal(
        size=(len(sc.cams), sc.height, sc.width, 4)).astype(np.float32)).cuda()
    ta, va = a.backward(g)
    tb, vb = b.backward(g)
    assert torch.allclose(ta, tb, rtol=1e-4, atol=1e-7 * float(tb.abs().max()))
    assert torch.allclose(va, vb, rtol=1e-4, atol=1e-6 * float(vb.abs().max()))
    a.release()
    b.release()


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16", "fp8"])
def test_cell_layout_every_storage(storage):
    """The cell layout's eight-corner decode for every storage type equals
    the eight-load path: identical frames on an uneven k-d partition."""
    dims = (44, 38, 34)
    cams = inputs.random_cameras(dims, 2, seed=31)
    sc = scenes.make(dims, kd=6, cams=cams, width=72, height=52, storage=storage, tile=(16, 8))
    imgs = []
    for gather in ("cell", "linear"):
        dev = scenes.gpu_device(sc, order=False)
        dev.set_frame(sc.width, sc.height, step_voxels=sc.step, sigma_max=sc.sigma_max, ert=sc.ert, tile=sc.tile,
                      gather=gather)
        dev.render()
        assert dev.stats()["error_flags"] == 0
        imgs.append([dev.map_frame(c)[0].clone() for c in range(len(sc.cams))])
        dev.release()
    for a, b in zip(*imgs):
        assert float(b[..., 3].max()) > 0.1
        assert torch.equal(a, b)
