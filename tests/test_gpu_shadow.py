"""GPU volumetric shadows by ray forwarding (DPV_FRAME_SHADOW) against the
FP64 oracle on the same stored values.

Every primary sample spawns a shadow ray toward the light; in K rounds each
brick marches every brick's wave-front through the shadow samples it owns;
the shading march scales each sample's emission by k_a + (1 - k_a) T_light.

* the frame within 1e-5 per channel of the oracle's partitioned render on
  every pixel the oracle does not flag (the sample count at the volume's
  exit, a shadow sample of opacity > 0 within 1e-3 node of the volume's
  faces, the opacity within 1e-4 of the termination threshold), regular
  and k-d partitions, a camera inside, f32 / f16 / bf16, several lights
  and shadow steps, early termination on and off;
* primary samples equal the oracle's up to the flagged pixels' rays; depth
  and opacity equal the unshadowed frame's bit for bit;
* k_a = 1 gives the unshadowed frame bit for bit; the three gather layouts
  agree bit for bit;
* refusals: the adjoint, the staged / iso / ordered / skipping / deep
  forms, a frame without a light, invalid lights.
"""
import numpy as np
import pytest
import torch

from paper_2407_00179_b300 import build, dpv, inputs

import scenes

pytestmark = pytest.mark.gpu

TOL = 1e-5

CASES = [
    dict(dims=(48, 40, 44), splits=(2, 2, 2), width=64, height=52, light=((0.3, 0.8, 0.5), 1.0, 0.25)),
    dict(dims=(50, 42, 36), kd=9, width=61, height=45, tile=(8, 4), storage="f16",
         light=((-0.7, 0.1, 0.7), 0.5, 0.1)),
    dict(dims=(50, 42, 36), kd=5, width=57, height=43, tile=(32, 8), inside=True,
         light=((0.0, 0.0, 1.0), 1.5, 0.3)),
    dict(dims=(40, 36, 32), splits=(2, 1, 2), width=52, height=44, storage="bf16", sigma_max=30.0, ert=0.95,
         light=((0.5, -0.6, -0.6), 1.0, 0.0)),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    dpv.load()


def _scene(i):
    c = dict(CASES[i])
    inside = c.pop("inside", False)
    dims = c.pop("dims")
    light = c.pop("light")
    cams = inputs.random_cameras(dims, 2, seed=110 + i, inside=inside)
    sc = scenes.make(dims, cams=cams, nblobs=10, seed=i, **c)
    sc.tf = inputs.make_tf(1234, transparent_below=0.05)
    return sc, light


def _device(sc, light, shadow=True, gather="auto"):
    dev = scenes.gpu_device(sc, order=False)
    if light is not None:
        dev.set_light(*light)
    dev.set_frame(sc.width, sc.height, step_voxels=sc.step, sigma_max=sc.sigma_max, ert=sc.ert, tile=sc.tile,
                  gather=gather, shadow=shadow)
    dev.reset_stats()
    dev.render()
    return dev


@pytest.mark.parametrize("i", range(len(CASES)))
def test_shadow_matches_fp64_oracle(orc, i):
    sc, light = _scene(i)
    dev = _device(sc, light)
    st = dev.stats()
    assert st["error_flags"] == 0
    assert st["samples_shadow"] > st["samples_forward"]
    plain = _device(sc, None, shadow=False)
    bricks = scenes.oracle_bricks(orc, sc)
    fr = scenes.oracle_frame(orc, sc)
    ol = orc.Light(light[0], step_voxels=light[1], ambient=light[2])
    n_ref = n_flag = 0
    worst = 0.0
    dark = 0
    for ci, cam in enumerate(sc.cams):
        ref = orc.render_shadow(sc.dims, sc.tf, cam, fr, ol, bricks=bricks, spacing=sc.spacing)
        rgba, depth = dev.map_frame(ci)
        prgba, pdepth = plain.map_frame(ci)
        assert torch.equal(rgba[..., 3], prgba[..., 3]) and torch.equal(depth, pdepth)
        rgba = rgba.reshape(-1, 4).double().cpu().numpy()
        amb = orc.FLAG_EXIT_AMBIG | orc.FLAG_ERT_AMBIG | orc.FLAG_SHADOW_AMBIG
        ok = (ref["flags"] & amb) == 0
        assert ok.mean() > 0.9
        err = np.abs(rgba - ref["rgba"])[ok]
        assert err.max() <= TOL, err.max()
        worst = max(worst, float(err.max()))
        dark += int((prgba.reshape(-1, 4)[:, :3].double().cpu().numpy() - rgba[:, :3] > 1e-3).sum())
        n_ref += int(ref["nsamples"].sum())
        n_flag += int(ref["nsamples"][~ok].sum())
    assert abs(st["samples_forward"] - n_ref) <= n_flag
    print("shadow case %d: max err %.2e, %d shadowed channels, %d shadow samples" % (
        i, worst, dark, st["samples_shadow"]))
    assert dark > 50
    dev.release()
    plain.release()


def test_full_ambient_is_unshadowed():
    sc, light = _scene(1)
    a = _device(sc, (light[0], light[1], 1.0))
    b = _device(sc, None, shadow=False)
    for c in range(len(sc.cams)):
        for x, y in zip(a.map_frame(c), b.map_frame(c)):
            assert torch.equal(x, y)
    a.release()
    b.release()


def test_shadow_layouts_agree():
    sc, light = _scene(0)
    frames = []
    for gather in ("cell", "quad", "linear"):
        dev = _device(sc, light, gather=gather)
        frames.append([t.clone() for c in range(len(sc.cams)) for t in dev.map_frame(c)])
        dev.release()
    for other in frames[1:]:
        for a, b in zip(frames[0], other):
            assert torch.equal(a, b)


def test_shadow_refusals():
    sc, light = _scene(0)
    dev = scenes.gpu_device(sc, order=False)
    dev.set_frame(sc.width, sc.height, shadow=True)
    with pytest.raises(dpv.DPVError, match="STATE"):
        dev.render()                                   # no light yet
    for bad in (((0.0, 0.0, 0.0), 1.0, 0.2), ((1.0, 0.0, 0.0), 0.0, 0.2), ((1.0, 0.0, 0.0), 1.0, 1.5)):
        with pytest.raises(dpv.DPVError, match="INVALID_ARG"):
            dev.set_light(*bad)
    dev.set_light(*light)
    dev.render()
    with pytest.raises(dpv.DPVError, match="UNSUPPORTED"):
        dev.backward(torch.zeros((len(sc.cams), sc.height, sc.width, 4), device="cuda"))
    for kw in (dict(iso=0.5), dict(ordered=True), dict(staged=True), dict(skip=True), dict(deep=True)):
        with pytest.raises(dpv.DPVError, match="UNSUPPORTED"):
            dev.set_frame(sc.width, sc.height, shadow=True, **kw)
    dev.release()
