"""Edge cases of the GPU path against the FP64 oracle.

* nothing in view (a camera looking away): no work item, an empty frame
  (zero RGBA, depth +inf), no sample, zero gradients -- in every mode
  (sort-last, skipping, deep fragments, ordered, iso-surface, shadows);
* images smaller than one tile (1 x 1, 3 x 2, 9 x 5);
* the smallest and largest TF tables (2 and 4096 entries): frames 1e-5
  and gradients within the adjoint bar, the TF gradient's widened by the
  oracle's TF-coordinate ambiguity: FP32 holds u = (s - vmin)(n - 1) /
  (vmax - vmin) to a few roundings of 2^-24 u, which moves the split of a
  sample's value adjoint between entries i0 and i0 + 1 -- at n = 4096 by
  up to 2.4e-4 of it (measured relative L2 before widening 1.1e-4);
* 240 bricks (15 x 4 x 4) of a small volume, so rays cross more bricks than
  the compositor sorts in registers: frame 1e-5, per-pixel order
  bit-exact;
* bricks one node thick (20 x 1 x 1 slabs).
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


def _away(dims):
    c = inputs.camera_from_direction(dims, (1.0, 0.7, 0.5))
    eye = np.asarray(c.eye)
    centre = np.asarray(c.center)
    return scenes.f32_camera(inputs.Camera(tuple(eye), tuple(eye + (eye - centre)), c.up, c.fovy_deg))


@pytest.mark.parametrize("mode", ["plain", "skip", "deep", "ordered", "iso", "shadow"])
def test_nothing_in_view(mode):
    dims = (40, 36, 32)
    sc = scenes.make(dims, splits=(2, 2, 2), cams=[_away(dims)], width=48, height=40)
    dev = scenes.gpu_device(sc, order=False)
    kw = {"plain": {}, "skip": dict(skip=True), "deep": dict(deep=True), "ordered": dict(ordered=True),
          "iso": dict(iso=0.5), "shadow": dict(shadow=True)}[mode]
    if mode == "shadow":
        dev.set_light((0.0, 1.0, 0.0))
    dev.set_frame(sc.width, sc.height, **kw)
    dev.reset_stats()
    dev.render()
    st = dev.stats()
    assert st["error_flags"] == 0 and st["work_items"] == 0 and st["samples_forward"] == 0
    rgba, depth = dev.map_frame(0)
    assert float(rgba.abs().max()) == 0.0
    assert bool(torch.isinf(depth).all())
    if mode == "plain":
        dtf, dvol = dev.backward(torch.ones((1, sc.height, sc.width, 4), device="cuda"))
        assert float(dtf.abs().max()) == 0.0 and float(dvol.abs().max()) == 0.0
    dev.release()


@pytest.mark.parametrize("size", [(1, 1), (3, 2), (9, 5)])
def test_images_smaller_than_a_tile(orc, size):
    dims = (30, 26, 28)
    cams = [scenes.f32_camera(inputs.camera_from_direction(dims, (0.8, -0.5, 0.3)))]
    sc = scenes.make(dims, kd=5, width=size[0], height=size[1], cams=cams)
    dev = scenes.gpu_device(sc, order=False)
    dev.render()
    ref = scenes.o_bricks(orc, sc, sc.cams[0])
    rgba = dev.map_frame(0)[0].reshape(-1, 4).double().cpu().numpy()
    ok = (ref["flags"] & (scenes.FLAG["exit"])) == 0
    assert ok.any() and ref["rgba"][ok, 3].max() > 0.2
    assert np.abs(rgba - ref["rgba"])[ok].max() <= TOL
    dev.release()


@pytest.mark.parametrize("ntf", [2, 4096])
def test_smallest_and_largest_tables(orc, ntf):
    dims = (36, 32, 30)
    cams = inputs.sphere_cameras(dims, 2, seed=6)
    sc = scenes.make(dims, splits=(2, 1, 2), nblobs=8, cams=cams, width=40, height=36)
    sc.tf = inputs.make_tf(4321, n=ntf)
    dev = scenes.gpu_device(sc, order=False)
    dev.render()
    bricks = scenes.oracle_bricks(orc, sc)
    fr = scenes.oracle_frame(orc, sc)
    g = inputs.rng(1, inputs.STREAM_GRAD).normal(size=(len(sc.cams), sc.height, sc.width, 4))
    rtf, rvol, avol, atf, ktf, kvol = 0.0, 0.0, 0.0, 0.0, 0.0, 0.0
    for ci, cam in enumerate(sc.cams):
        ref = orc.render_bricks(sc.dims, bricks, sc.tf, cam, fr, spacing=sc.spacing)
        rgba = dev.map_frame(ci)[0].reshape(-1, 4).double().cpu().numpy()
        ex = (ref["flags"] & (scenes.FLAG["exit"] | scenes.FLAG["ert"] | scenes.FLAG["owner"])) != 0
        assert np.abs(rgba - ref["rgba"])[~ex].max() <= TOL
        g[ci].reshape(-1, 4)[ex] = 0.0
        gi = g[ci].reshape(-1, 4).astype(np.float32).astype(np.float64)
        a, b, amb, tamb = orc.grad_bricks(sc.dims, bricks, sc.tf, cam, fr, gi, spacing=sc.spacing,
                                          knot_eps=orc.KNOT_EPS, tf_amb=True)
        rtf, rvol, avol, atf = rtf + a, rvol + b, avol + amb, atf + tamb
        for eps in (1e-7, -1e-7):
            pa, pb = orc.grad_bricks(sc.dims, bricks, sc.tf, scenes.perturbed_eye(cam, eps), fr, gi,
                                     spacing=sc.spacing)
            ktf = np.maximum(ktf, np.abs(pa - a))
            kvol = np.maximum(kvol, np.abs(pb - b))
    dtf, dvol = dev.backward(torch.from_numpy(g.astype(np.float32)).cuda())
    assert dtf.shape == (ntf, 4)
    l2a, va = scenes.grad_checks(dtf.cpu().numpy(), rtf, "dL/dTF", ktf, atf)
    l2b, vb = scenes.grad_checks(dvol.double().cpu().numpy(), rvol, "dL/dvolume", kvol, avol)
    assert l2a <= 1e-4 and l2b <= 1e-4, (l2a, l2b)
    assert va == 0 and vb == 0, (va, vb)
    dev.release()


def test_more_bricks_along_a_ray_than_sorted_in_registers(orc):
    dims = (40, 38, 36)
    cams = [scenes.f32_camera(inputs.camera_from_direction(dims, (1.0, 0.35, 0.3)))]
    sc = scenes.make(dims, splits=(15, 4, 4), nblobs=12, cams=cams, width=40, height=36)
    dev = scenes.gpu_device(sc, order=True)
    dev.render()
    K = sc.part.num_ranks
    assert K == 240
    bricks = scenes.oracle_bricks(orc, sc)
    ref = orc.render_bricks(sc.dims, bricks, sc.tf, sc.cams[0], scenes.oracle_frame(orc, sc), spacing=sc.spacing)
    rgba = dev.map_frame(0)[0].reshape(-1, 4).double().cpu().numpy()
    ok = (ref["flags"] & (scenes.FLAG["exit"] | scenes.FLAG["owner"])) == 0
    assert np.abs(rgba - ref["rgba"])[ok].max() <= TOL
    order = dev.order(0).reshape(-1, K).cpu().numpy()
    np.testing.assert_array_equal(order[ok], ref["order"][ok])
    nfrag = (ref["frag_key"] != 2 ** 31 - 1).sum(axis=1)
    assert nfrag[ok].max() > 16                       # the fallback past the register sort ran
    dev.release()


def test_bricks_one_node_thick(orc):
    dims = (20, 18, 16)
    sc = scenes.make(dims, splits=(20, 1, 1), nblobs=6, width=32, height=28)
    dev = scenes.gpu_device(sc, order=True)
    dev.render()
    ref = scenes.o_bricks(orc, sc, sc.cams[0])
    rgba = dev.map_frame(0)[0].reshape(-1, 4).double().cpu().numpy()
    ok = (ref["flags"] & (scenes.FLAG["exit"] | scenes.FLAG["owner"])) == 0
    assert np.abs(rgba - ref["rgba"])[ok].max() <= TOL
    order = dev.order(0).reshape(-1, sc.part.num_ranks).cpu().numpy()
    np.testing.assert_array_equal(order[ok], ref["order"][ok])
    dev.release()
