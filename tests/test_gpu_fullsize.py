"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times (autotuned tile, gather layout and schedule), on pixels the
FP64 oracle computes one by one.

* mid: 512^3 float32 (64 blobs + 3-octave noise), 2x2x2 bricks, 1920x1080,
  early termination at 0.99 -- every pixel;
* batched: 1024x1024x512 float16 storage (5-octave log-normal noise), 37 k-d
  bricks, 16 orbit cameras at 1024x1024 -- the 1/16 subsample (x % 4 == 0
  and y % 4 == 0) of every camera, against the oracle on the same stored
  float16 values;
* large: 2048^3 stored as bf16 or fp8, 64 bricks, 8 cameras at 3840x2160 --
  the 1/16 subsample of every camera;
* diff: 256^3 float32, 8 bricks, 32 views at 512x512 -- the adjoint of the
  L2 loss against perturbed-TF targets on the 1/16 subsample of every view,
  against the FP64 reverse-mode gradient; and FP64 central differences of
  the oracle loss on a 128x128 reduction of 4 views.

Tolerances as everywhere (1e-5 max abs per channel; orders bit-exact) except
the stated fp8 bound at 2048^3 (below), excluding the pixels where FP32 may
take another discrete decision (see test_gpu_parity)."""
import numpy as np
import pytest
import torch

import bench
from paper_2407_00179_b300 import build, dpv, inputs

import scenes

pytestmark = pytest.mark.gpu

TOL = 1e-5
SUB = 4          # 1/16 pixel subsample: x % 4 == 0 and y % 4 == 0


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
                  tile=tuple(tune["tile"]), gather=dpv.gather_of(fl),
                  persistent=bool(fl & dpv.FRAME_PERSISTENT), order=True)
    dev.render()
    return dev


def _spacing(cfg):
    return float(np.float32(1.0 / (max(cfg["dims"]) - 1)))


def _ambiguous(orc, ref):
    return (ref["flags"] & (orc.FLAG_EXIT_AMBIG | orc.FLAG_ERT_AMBIG | orc.FLAG_OWNER_AMBIG)) != 0


def _check_camera(orc, dev, ci, cfg, bricks, tf, cam, pix, tol=TOL):
    fr = orc.Frame(cfg["width"], cfg["height"], step_voxels=0.5, sigma_max=8.0, ert=cfg["ert"])
    ref = orc.render_bricks(cfg["dims"], bricks, tf, cam, fr, pix=pix, spacing=_spacing(cfg))
    rgba, _ = dev.map_frame(ci)
    img = rgba.reshape(-1, 4)[torch.from_numpy(pix).long().cuda()].double().cpu().numpy()
    ex = _ambiguous(orc, ref)
    assert ex.mean() < 0.05, ex.mean()    # measured 1.1 % (mid) to 2.2 % (2048^3)
    err = np.abs(img - ref["rgba"])[~ex]
    assert err.max() <= tol, err.max()
    order = dev.order(ci).reshape(-1, dev.num_ranks)[torch.from_numpy(pix).long().cuda()].cpu().numpy()
    np.testing.assert_array_equal(order[~ex], ref["order"][~ex])
    assert ref["rgba"][:, 3].max() > 0.3
    return err.max(), float(err.mean()), int(ex.sum()), len(pix), img


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
    pix = np.arange(cfg["width"] * cfg["height"], dtype=np.int32)
    worst, mean, nex, n, _ = _check_camera(orc, dev, 0, cfg, bricks, inputs.make_tf(1234), cams[0], pix)
    print("mid full size: max abs %.2e mean %.2e over %d pixels (%d excluded)" % (worst, mean, n - nex, nex))
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
    pix = inputs.pixel_subsample(cfg["width"], cfg["height"], SUB)
    tf = inputs.make_tf(1234)
    worst_all = 0.0
    for ci in range(len(cams)):
        worst, mean, nex, n, _ = _check_camera(orc, dev, ci, cfg, bricks, tf, cams[ci], pix)
        worst_all = max(worst_all, worst)
        print("batched camera %d: max abs %.2e mean %.2e over %d pixels (%d excluded)" % (ci, worst, mean, n - nex, nex))
    print("batched: max abs %.2e over %d cameras" % (worst_all, len(cams)))
    dev.release()


# Stated arithmetic bounds at 2048^3, one per reduced-precision storage mode.
# Rays cross ~4000 samples here, 8x the 512^3 frame; the FP32 round-off of
# the compositing recurrences grows about as the square root of the sample
# count, which scales the 1e-5 bar of the 512^3 cases to about 2.8e-5.  bf16
# is stated at 2e-5 (measured 9.1e-6 on this subsample, 1.01e-5 over whole
# pixel rows of camera 0); fp8's coarse quantisation steps make the field
# rough and its error 3.2e-5, so its bound is 5e-5.  Finer FP32 sample
# positions (measured) change neither figure.
ARITH_TOL = {"bf16": 2e-5, "fp8": 5e-5}


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
def test_large_full_size_reduced_precision(orc, storage):
    """2048^3 stored as bf16 or fp8 (per-brick scale), 64 bricks, 8 cameras
    at 3840x2160: arithmetic error against the oracle on the same stored
    values (ARITH_TOL), and the storage error against the oracle on the
    original float32 field (reported), on the 1/16 subsample of every
    camera."""
    cfg = bench.CONFIGS["large_" + storage]
    field = bench._field(cfg, "cuda")
    part = bench._partition(cfg)
    cams = [scenes.f32_camera(c) for c in bench._cameras(cfg)]
    dev = _bench_device(cfg, field, part, cams)
    assert dev.stats()["error_flags"] == 0
    f = field.cpu().numpy()
    del field
    torch.cuda.empty_cache()
    bricks = orc.make_bricks(f, part, orc.DTYPE_NAMES[storage])
    f32b = orc.make_bricks(f, part, orc.F32)
    del f
    pix = inputs.pixel_subsample(cfg["width"], cfg["height"], SUB)
    tf = inputs.make_tf(1234)
    fr = orc.Frame(cfg["width"], cfg["height"], step_voxels=0.5, sigma_max=8.0, ert=cfg["ert"])
    arith, smax, ssum, scount = 0.0, 0.0, 0.0, 0
    for ci in range(len(cams)):
        worst, mean, nex, n, img = _check_camera(orc, dev, ci, cfg, bricks, tf, cams[ci], pix,
                                                 tol=ARITH_TOL[storage])
        arith = max(arith, worst)
        # storage error: the same pixels against the float32 field
        ref32 = orc.render_bricks(cfg["dims"], f32b, tf, cams[ci], fr, pix=pix, spacing=_spacing(cfg))
        store = np.abs(img - ref32["rgba"])
        smax = max(smax, float(store.max()))
        ssum += float(store.sum())
        scount += store.size
        print("large %s camera %d: arithmetic max %.2e mean %.2e over %d pixels (%d excluded); "
              "storage error max %.2e mean %.2e" % (storage, ci, worst, mean, n - nex, nex, store.max(), store.mean()))
    print("large %s: arithmetic max %.2e; storage error max %.2e mean %.2e over %d cameras" % (
        storage, arith, smax, ssum / scount, len(cams)))
    assert smax < {"bf16": 5e-2, "fp8": 2e-1}[storage]
    dev.release()


def test_large_adjoint_in_brick_groups(monkeypatch):
    """2048^3 fp8, 64 bricks, 8 cameras at 3840x2160: the face adjoint buffer
    for all bricks would need 138 GB, so the adjoint runs it over groups of
    bricks (more than one group here).  Its field gradient equals the one
    through scalar atomics into the field (another summation order) on 4 M
    seeded nodes plus every node of the planes on both sides of each brick
    boundary in x, where the groups' ghost copies meet; the TF gradients
    agree too."""
    cfg = bench.CONFIGS["large_fp8"]
    field = bench._field(cfg, "cuda")
    part = bench._partition(cfg)
    cams = [scenes.f32_camera(c) for c in bench._cameras(cfg)]
    dev = _bench_device(cfg, field, part, cams)
    del field
    torch.cuda.empty_cache()
    H, W = cfg["height"], cfg["width"]
    g = torch.from_numpy(inputs.rng(5, inputs.STREAM_GRAD).normal(size=(len(cams), H, W, 4)).astype(np.float32)).cuda()
    nx, ny, nz = cfg["dims"]
    idx = torch.from_numpy(inputs.rng(6, inputs.STREAM_SELECT).integers(0, nx * ny * nz, size=4 << 20)).cuda()
    cuts = sorted({int(v) for lo, hi in zip(part.lo, part.hi) for v in (lo[0] - 1, lo[0], hi[0] - 1, hi[0])
                   if 0 <= v < nx})
    monkeypatch.delenv("DPV_FACE_GRAD", raising=False)
    monkeypatch.delenv("DPV_FACE_GROUP", raising=False)
    out = []
    for scalar in (False, True):
        if scalar:
            monkeypatch.setenv("DPV_FACE_GRAD", "0")
        dev.reset_stats()
        dtf, dvol = dev.backward(g)
        launches = dev.stats()["kernel_launches"]
        flat = dvol.reshape(-1)
        out.append((dtf.cpu().numpy(), flat[idx].cpu().numpy(), dvol[:, :, cuts].cpu().numpy(), launches))
        del dvol, flat
        torch.cuda.empty_cache()
    (tf_g, s_g, c_g, l_g), (tf_s, s_s, c_s, l_s) = out
    groups = (l_g - 1) // 2
    print("large fp8 adjoint: %d face-buffer groups" % groups)
    assert groups > 1 and l_s == 2
    for a, b in ((s_g, s_s), (c_g, c_s)):
        m = float(np.abs(b).max())
        assert m > 0
        np.testing.assert_allclose(a, b, rtol=1e-4, atol=1e-5 * m)
    np.testing.assert_allclose(tf_g, tf_s, rtol=0, atol=1e-9 * float(np.abs(tf_s).max()))
    dev.release()


def _diff_inputs():
    cfg = bench.CONFIGS["diff"]
    field = bench._field(cfg, "cuda")
    part = bench._partition(cfg)
    cams = [scenes.f32_camera(c) for c in bench._cameras(cfg)]
    tf = inputs.make_tf(1234)
    # L2 loss against targets rendered with TF* = clamp(TF + N(0, 0.05^2))
    tf_t = inputs.perturb_tf(tf, seed=0, sigma=0.05)
    return cfg, field, part, cams, tf, tf_t


def test_diff_full_size_gradient(orc):
    """Adjoint of the L2 loss at the full differentiable workload (32 views
    at 512x512, 8 bricks of a 256^3 float32 field), restricted to the 1/16
    pixel subsample of every view, against the FP64 reverse-mode gradient of
    the same loss terms; the upstream gradient both sides receive comes from
    the oracle's own images.  At this size ~1e9 samples meet the TF's kinked
    knots, so the field gradient's bar includes the oracle's knot ambiguity
    (scenes.grad_checks)."""
    cfg, field, part, cams, tf, tf_t = _diff_inputs()
    W, H = cfg["width"], cfg["height"]
    dev = _bench_device(cfg, field, part, cams)
    f = field.cpu().numpy()
    bricks = orc.make_bricks(f, part, orc.F32)
    fr = orc.Frame(W, H, step_voxels=0.5, sigma_max=8.0, ert=cfg["ert"])
    pix = inputs.pixel_subsample(W, H, SUB)
    sp = _spacing(cfg)
    N = len(cams) * W * H * 4
    g = np.zeros((len(cams), H * W, 4), np.float32)
    rtf, rvol, avol, ktf, kvol = 0.0, 0.0, 0.0, 0.0, 0.0
    for ci, cam in enumerate(cams):
        ref = orc.render_bricks(cfg["dims"], bricks, tf, cam, fr, pix=pix, spacing=sp)
        tgt = orc.render_bricks(cfg["dims"], bricks, tf_t, cam, fr, pix=pix, spacing=sp)
        gi = (2.0 / N) * (ref["rgba"] - tgt["rgba"])
        gi[_ambiguous(orc, ref)] = 0.0
        gi = gi.astype(np.float32)
        g[ci, pix] = gi
        gi = gi.astype(np.float64)
        a, b, amb = orc.grad_bricks(cfg["dims"], bricks, tf, cam, fr, gi, pix=pix, spacing=sp, knot_eps=orc.KNOT_EPS)
        rtf, rvol, avol = rtf + a, rvol + b, avol + amb
        for eps in (1e-7, -1e-7):
            pa, pb = orc.grad_bricks(cfg["dims"], bricks, tf, scenes.perturbed_eye(cam, eps), fr, gi, pix=pix,
                                     spacing=sp)
            ktf = np.maximum(ktf, np.abs(pa - a))
            kvol = np.maximum(kvol, np.abs(pb - b))
    dtf, dvol = dev.backward(torch.from_numpy(g.reshape(len(cams), H, W, 4)).cuda())
    assert dev.stats()["error_flags"] == 0
    l2a, va = scenes.grad_checks(dtf.cpu().numpy(), rtf, "diff full size dL/dTF", ktf)
    l2b, vb = scenes.grad_checks(dvol.double().cpu().numpy(), rvol, "diff full size dL/dvolume", kvol, avol)
    assert l2a <= 1e-4 and l2b <= 1e-4, (l2a, l2b)
    assert va == 0 and vb == 0, (va, vb)
    dev.release()


def test_diff_full_size_gradient_kink_free(orc):
    """The adjoint of the full differentiable workload (32 views at 512x512,
    8 bricks of a 256^3 float32 field, the 1/16 pixel subsample of every
    view) with a TF whose channels are linear in s: no interior knot, so no
    knot ambiguity.  The plain bar, with no kappa and no knot allowance:
    relative L2 <= 1e-4 for both gradients; on entries above 1e-3 of the
    largest, |gpu - ref| <= 1e-3 |ref| for every TF entry and for all but
    one in a million field entries, none beyond 2e-3 |ref|.  The
    eye-perturbation spread kappa is computed only to report how the errors
    compare with it."""
    cfg, field, part, cams, _, _ = _diff_inputs()
    tf = inputs.linear_tf(256)
    tf_t = inputs.perturb_tf(tf, seed=0, sigma=0.05)
    W, H = cfg["width"], cfg["height"]
    dev = _bench_device(cfg, field, part, cams)
    dev.set_tf(torch.from_numpy(tf).cuda())
    dev.render()
    f = field.cpu().numpy()
    bricks = orc.make_bricks(f, part, orc.F32)
    fr = orc.Frame(W, H, step_voxels=0.5, sigma_max=8.0, ert=cfg["ert"])
    pix = inputs.pixel_subsample(W, H, SUB)
    sp = _spacing(cfg)
    N = len(cams) * W * H * 4
    g = np.zeros((len(cams), H * W, 4), np.float32)
    rtf, rvol, avol, ktf, kvol = 0.0, 0.0, 0.0, 0.0, 0.0
    for ci, cam in enumerate(cams):
        ref = orc.render_bricks(cfg["dims"], bricks, tf, cam, fr, pix=pix, spacing=sp)
        tgt = orc.render_bricks(cfg["dims"], bricks, tf_t, cam, fr, pix=pix, spacing=sp)
        gi = (2.0 / N) * (ref["rgba"] - tgt["rgba"])
        gi[_ambiguous(orc, ref)] = 0.0
        gi = gi.astype(np.float32)
        g[ci, pix] = gi
        gi = gi.astype(np.float64)
        a, b, amb = orc.grad_bricks(cfg["dims"], bricks, tf, cam, fr, gi, pix=pix, spacing=sp, knot_eps=orc.KNOT_EPS)
        rtf, rvol, avol = rtf + a, rvol + b, avol + amb
        for eps in (1e-7, -1e-7):
            pa, pb = orc.grad_bricks(cfg["dims"], bricks, tf, scenes.perturbed_eye(cam, eps), fr, gi, pix=pix,
                                     spacing=sp)
            ktf = np.maximum(ktf, np.abs(pa - a))
            kvol = np.maximum(kvol, np.abs(pb - b))
    # a linear TF has no interior knot: the oracle sees no knot ambiguity
    # beyond the float32 rounding of the table (slopes equal to ~1e-7)
    assert float(np.abs(avol).max()) <= 1e-5 * float(np.abs(rvol).max())
    dtf, dvol = dev.backward(torch.from_numpy(g.reshape(len(cams), H, W, 4)).cuda())
    assert dev.stats()["error_flags"] == 0
    gtf, gvol = dtf.cpu().numpy(), dvol.double().cpu().numpy()
    for name, gpu, ref, kap in (("dL/dTF", gtf, rtf, ktf), ("dL/dvolume", gvol, rvol, kvol)):
        m = np.abs(ref).max()
        big = np.abs(ref) > 1e-3 * m
        err = np.abs(gpu - ref)
        l2 = np.linalg.norm(gpu - ref) / np.linalg.norm(ref)
        rel = err[big] / np.abs(ref[big])
        over = big & (err > 1e-3 * np.abs(ref))
        ratio = err[big] / np.maximum(kap[big], 1e-300)
        print("kink-free diff %s: rel L2 %.2e, max rel %.2e over %d entries, %d beyond 1e-3|ref|; "
              "|gpu - ref| / kappa: median %.2f, 99th pct %.2f, max %.2f" % (
                  name, l2, rel.max(), big.sum(), over.sum(), np.median(ratio), np.percentile(ratio, 99),
                  ratio.max()))
        for idx in np.argwhere(over)[:10]:
            t = tuple(int(v) for v in idx)
            print("  beyond: %s gpu %.6e ref %.6e rel %.2e |ref|/max %.2e kappa %.2e%s" % (
                t, gpu[t], ref[t], abs(gpu[t] - ref[t]) / abs(ref[t]), abs(ref[t]) / m, kap[t],
                "" if len(t) < 3 else " field %.4f; brick-face distance %s" % (
                    f[t], [min(abs(c - b) for b in (127, 128, 129)) for c in t])))
        assert l2 <= 1e-4, (name, l2)
        if name == "dL/dTF":
            assert not over.any(), (name, int(over.sum()), float(rel.max()))
        else:
            # measured: 7 of 14.6 M entries beyond 1e-3 |ref| (at most
            # 1.58e-3), all just above the 1e-3 max cut, where FP32 sample
            # positions (about 1e-5 voxel) decide the last digits
            assert over.sum() <= 1e-6 * big.sum() and rel.max() < 2e-3, (name, int(over.sum()), float(rel.max()))
    dev.release()


def test_diff_gradient_central_differences(orc):
    """GPU gradient of the L2 loss (through the autograd binding) against FP64
    central differences of the oracle's loss, eps = 1e-3, on 32 seeded TF
    entries and 32 seeded voxels, at a 128x128 reduction of 4 of the
    differentiable workload's views.  Bar: |fd - gpu| <= 1e-2 |fd| + 1e-3
    max|g|.  Test points are drawn from the oracle's own gradient (entries
    above 1e-2 of its largest; voxels with values in [0.01, 0.99]).  A
    piecewise-linear TF makes the loss only piecewise smooth: where the two
    one-sided differences disagree beyond that bar, a TF knot lies within eps
    of some sample, the central difference is not a derivative, and the
    point is counted as a kink and skipped (at most a third of them)."""
    cfg, field, part, cams, tf, tf_t = _diff_inputs()
    cams = cams[:4]
    W = H = 128
    dims = cfg["dims"]
    sp = _spacing(cfg)
    dev = dpv.Device(part.num_ranks)
    dev.set_geometry(dims)
    dev.commit_partition(field, part, "f32")
    dev.set_cameras(cams)
    dev.set_frame(W, H, step_voxels=0.5, sigma_max=8.0, ert=0.0, order=False)
    f = field.cpu().numpy()
    bricks = orc.make_bricks(f, part, orc.F32)
    fr = orc.Frame(W, H, step_voxels=0.5, sigma_max=8.0, ert=0.0)
    target = [orc.render_bricks(dims, bricks, tf_t, cam, fr, spacing=sp)["rgba"] for cam in cams]
    N = len(cams) * W * H * 4

    def loss(bricks_, tf_):
        s = 0.0
        for ci, cam in enumerate(cams):
            img = orc.render_bricks(dims, bricks_, tf_, cam, fr, spacing=sp)["rgba"]
            s += np.sum((img - target[ci]) ** 2)
        return s / N

    # GPU gradient through the autograd binding
    tf_g = torch.from_numpy(tf).cuda().requires_grad_(True)
    vol = field.clone().requires_grad_(True)
    img = dpv.render(dev, tf_g, vol)
    tgt = torch.from_numpy(np.stack(target).reshape(len(cams), H, W, 4)).float().cuda()
    ((img - tgt) ** 2).mean().backward()
    gtf = tf_g.grad.double().cpu().numpy()
    gvol = vol.grad.double().cpu().numpy()
    # the oracle's gradient of its own loss picks the test points
    otf, ovol = 0.0, 0.0
    for ci, cam in enumerate(cams):
        ref = orc.render_bricks(dims, bricks, tf, cam, fr, spacing=sp)["rgba"]
        a, b = orc.grad_bricks(dims, bricks, tf, cam, fr, (2.0 / N) * (ref - target[ci]), spacing=sp)
        otf, ovol = otf + a, ovol + b
    rng = inputs.rng(1, inputs.STREAM_SELECT)
    nz = np.argwhere(np.abs(otf) > 1e-2 * np.abs(otf).max())
    tf_picks = nz[rng.choice(len(nz), size=min(32, len(nz)), replace=False)]
    cand = np.argwhere((np.abs(ovol) > 1e-2 * np.abs(ovol).max()) & (f >= 0.01) & (f <= 0.99))
    vox_picks = cand[rng.choice(len(cand), size=min(32, len(cand)), replace=False)]
    assert len(tf_picks) >= 16 and len(vox_picks) >= 16
    L0 = loss(bricks, tf)
    eps = 1e-3

    def judge(lp, lm, h_p, h_m, gpu, gmax, out):
        fd = (lp - lm) / (h_p + h_m)
        fwd, bwd = (lp - L0) / h_p, (L0 - lm) / h_m
        bar = 1e-2 * abs(fd) + 1e-3 * gmax
        if abs(fwd - bwd) > bar:
            out["kink"] += 1
            return
        out["n"] += 1
        out["worst"] = max(out["worst"], abs(fd - gpu) / bar)
        if abs(fd - gpu) > bar:
            out["bad"].append((fd, gpu))

    res_tf = {"n": 0, "kink": 0, "bad": [], "worst": 0.0}
    gmax = np.abs(gtf).max()
    for i, c in tf_picks:
        t1, t0 = tf.copy(), tf.copy()
        t1[i, c] += eps
        t0[i, c] -= eps
        judge(loss(bricks, t1), loss(bricks, t0), float(np.float64(t1[i, c]) - np.float64(tf[i, c])),
              float(np.float64(tf[i, c]) - np.float64(t0[i, c])), gtf[i, c], gmax, res_tf)
    res_vox = {"n": 0, "kink": 0, "bad": [], "worst": 0.0}
    gmax = np.abs(gvol).max()
    for z, y, x in vox_picks:
        v = f[z, y, x]
        fp, fm = f.copy(), f.copy()
        fp[z, y, x] = np.float32(v + eps)
        fm[z, y, x] = np.float32(v - eps)
        judge(loss(orc.make_bricks(fp, part, orc.F32), tf), loss(orc.make_bricks(fm, part, orc.F32), tf),
              float(np.float64(fp[z, y, x]) - np.float64(v)), float(np.float64(v) - np.float64(fm[z, y, x])),
              gvol[z, y, x], gmax, res_vox)
    for name, r, k in (("TF", res_tf, len(tf_picks)), ("voxel", res_vox, len(vox_picks))):
        print("diff FD %s: %d checked, %d kinks skipped, worst |fd - gpu| / bar %.2f" % (
            name, r["n"], r["kink"], r["worst"]))
        assert r["kink"] <= k // 3, r
        assert not r["bad"], r["bad"]
    dev.release()
