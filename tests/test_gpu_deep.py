"""GPU deep fragments (DPV_FRAME_DEEP) against the FP64 oracle on the same
stored values.

Empty-space skipping splits each brick's ray segment at its transparent
macro-cells; every run of evaluated samples is a fragment (up to
DPV_DEEP_MAX per brick and pixel) and the compositor sorts the variable
count per pixel.

* per brick and layer: fragment keys bit-exact and fragment RGBA within
  1e-5, fragment counts equal, on every pixel the oracle does not flag (the
  sample count at the volume's exit, a sample near an internal brick face,
  a sample within 1e-3 node of a face between macro-cells of different
  transparency or a macro-cell range at a TF entry boundary, the opacity
  within 1e-4 of the termination threshold);
* the composited frame within 1e-5 of the oracle, depth 1e-5 relative, and
  within 1e-5 of the same frame without deep fragments;
* the order image lists, per pixel, the brick of every fragment in key
  order;
* evaluated samples equal the oracle's up to the flagged pixels' rays;
* the adjoint and the staged, iso-surface and ordered forms refuse deep
  frames; a layer past DPV_DEEP_MAX is an invalid argument.
"""
import numpy as np
import pytest
import torch

from paper_2407_00179_b300 import build, dpv, inputs

import scenes

pytestmark = pytest.mark.gpu

TOL = 1e-5
EMPTY = 2 ** 31 - 1

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


def _scene(i):
    c = dict(CASES[i])
    inside = c.pop("inside", False)
    dims = c.pop("dims")
    cams = inputs.random_cameras(dims, 2, seed=90 + i, inside=inside)
    sc = scenes.make(dims, cams=cams, nblobs=10, seed=i, **c)
    sc.tf = inputs.make_tf(1234, transparent_below=0.35)
    return sc


def _device(sc, deep=True, skip=False, order=True):
    dev = scenes.gpu_device(sc, order=False)
    dev.set_frame(sc.width, sc.height, step_voxels=sc.step, sigma_max=sc.sigma_max, ert=sc.ert, tile=sc.tile,
                  deep=deep, skip=skip, order=order)
    dev.reset_stats()
    dev.render()
    return dev


@pytest.mark.parametrize("i", range(len(CASES)))
def test_deep_matches_fp64_oracle(orc, i):
    sc = _scene(i)
    dev = _device(sc)
    st = dev.stats()
    assert st["error_flags"] == 0
    ref_dev = _device(sc, deep=False, skip=True, order=False)
    bricks = scenes.oracle_bricks(orc, sc)
    fr = scenes.oracle_frame(orc, sc)
    K, D = sc.part.num_ranks, dpv.DEEP_MAX
    n_ref = n_flag = split = 0
    for ci, cam in enumerate(sc.cams):
        ref = orc.render_deep(sc.dims, bricks, sc.tf, cam, fr, deep=D, spacing=sc.spacing)
        sl = orc.render_bricks(sc.dims, bricks, sc.tf, cam, fr, spacing=sc.spacing)
        rgba, depth = dev.map_frame(ci)
        rgba = rgba.reshape(-1, 4).double().cpu().numpy()
        depth = depth.reshape(-1).double().cpu().numpy()
        # the composite: values do not depend on how segments split
        amb_f = orc.FLAG_EXIT_AMBIG | orc.FLAG_ERT_AMBIG | (orc.FLAG_OWNER_AMBIG if sc.storage == "fp8" else 0)
        okf = (ref["flags"] & amb_f) == 0
        assert okf.mean() > 0.9
        assert np.abs(rgba - ref["rgba"])[okf].max() <= TOL
        other = ref_dev.map_frame(ci)[0].reshape(-1, 4).double().cpu().numpy()
        assert np.abs(rgba - other).max() <= TOL
        # fragments, keys, counts and depth: the split must agree
        amb = amb_f | orc.FLAG_OWNER_AMBIG | orc.FLAG_MACRO_AMBIG
        ok = (ref["flags"] & amb) == 0
        assert ok.mean() > 0.85
        count = np.zeros((ok.size, K), np.int64)
        for b in range(K):
            for layer in range(D):
                fr_rgba, fr_key = dev.read_fragments(ci, b, layer)
                key = fr_key.reshape(-1).cpu().numpy()
                np.testing.assert_array_equal(key[ok], ref["frag_key"][ok, b, layer])
                live = ok & (key != EMPTY)
                count[:, b] += key != EMPTY
                fr_rgba = fr_rgba.reshape(-1, 4).double().cpu().numpy()
                if live.any():
                    assert np.abs(fr_rgba[live] - ref["frag_rgba"][live, b, layer]).max() <= TOL
        np.testing.assert_array_equal(count[ok], ref["frag_count"][ok])
        split += int((ref["frag_count"][ok] > 1).sum())
        fin = ok & np.isfinite(ref["depth"])
        np.testing.assert_array_equal(np.isinf(depth[ok]), np.isinf(ref["depth"][ok]))
        if fin.any():
            assert np.abs(depth[fin] - ref["depth"][fin]).max() <= 1e-5 * np.abs(ref["depth"][fin]).max()
        # the order image: the brick of every fragment, in key order
        order = dev.order(ci).reshape(-1, K * D).cpu().numpy()
        for p in np.flatnonzero(ok)[::7]:
            fk = [(ref["frag_key"][p, b, l], b) for b in range(K) for l in range(D)
                  if ref["frag_key"][p, b, l] != EMPTY]
            want = [b for _, b in sorted(fk)] + [0xFF] * (K * D - len(fk))
            np.testing.assert_array_equal(order[p], want)
        n_ref += int(ref["nsamples"].sum())
        n_flag += int(sl["nsamples"][~ok].sum())
        assert ref["rgba"][:, 3].max() > 0.02
    assert abs(st["samples_forward"] - n_ref) <= n_flag
    print("deep case %d: %d brick segments split" % (i, split))
    assert split > 0
    dev.release()
    ref_dev.release()


def test_deep_layouts_and_schedules_agree():
    sc = _scene(1)
    frames = []
    for gather in ("cell", "quad", "linear"):
        for persistent in (False, True):
            dev = scenes.gpu_device(sc, order=False)
            dev.set_frame(sc.width, sc.height, step_voxels=sc.step, sigma_max=sc.sigma_max, ert=sc.ert,
                          tile=sc.tile, gather=gather, persistent=persistent, deep=True)
            dev.render()
            out = []
            for c in range(len(sc.cams)):
                out += [t.clone() for t in dev.map_frame(c)]
                for b in range(sc.part.num_ranks):
                    for layer in range(dpv.DEEP_MAX):
                        out += [t.clone() for t in dev.read_fragments(c, b, layer)]
            frames.append(out)
            dev.release()
    for other in frames[1:]:
        for a, b in zip(frames[0], other):
            assert torch.equal(a, b)


def test_deep_refusals():
    sc = _scene(0)
    dev = _device(sc, order=False)
    with pytest.raises(dpv.DPVError, match="UNSUPPORTED"):
        dev.backward(torch.zeros((len(sc.cams), sc.height, sc.width, 4), device="cuda"))
    with pytest.raises(dpv.DPVError, match="INVALID_ARG"):
        dev.read_fragments(0, 0, dpv.DEEP_MAX)
    for kw in (dict(iso=0.5), dict(ordered=True), dict(staged=True)):
        with pytest.raises(dpv.DPVError, match="UNSUPPORTED"):
            dev.set_frame(sc.width, sc.height, deep=True, **kw)
    dev.release()
    # without deep fragments only layer 0 exists
    dev = _device(sc, deep=False, order=False)
    with pytest.raises(dpv.DPVError, match="INVALID_ARG"):
        dev.read_fragments(0, 0, 1)
    dev.release()
