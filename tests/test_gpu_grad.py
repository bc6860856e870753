"""GPU adjoint parity (compositor + ray-march replay) against the FP64 oracle
gradient and against FP64 central finite differences of the oracle forward.

Tolerances: GPU vs FP64 gradient, max relative error 1e-3 on entries
above 1e-3 of the largest, relative L2 1e-4, each widened by the oracle's
geometric conditioning and, for the field gradient, its TF-knot ambiguity
(see scenes.grad_checks); GPU vs central differences with
eps = 1e-3 on 64 seeded TF entries, relative 1e-2 with an absolute floor of
1e-3 of the largest gradient."""
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


def _scene(ert=0.0, storage="f32"):
    dims = (40, 36, 32)
    cams = inputs.sphere_cameras(dims, 2, seed=4)
    sc = scenes.make(dims, splits=(2, 2, 2), nblobs=10, cams=cams, width=48, height=40, ert=ert, storage=storage)
    return sc


@pytest.mark.parametrize("ert", [0.0, 0.95])
def test_gradients_match_fp64_oracle(orc, ert):
    sc = _scene(ert=ert)
    dev = scenes.gpu_device(sc, order=False)
    dev.render()
    g = inputs.rng(0, inputs.STREAM_GRAD).normal(size=(len(sc.cams), sc.height, sc.width, 4))
    bricks = scenes.oracle_bricks(orc, sc)
    fr = scenes.oracle_frame(orc, sc)
    rtf, rvol, avol = 0.0, 0.0, 0.0
    ktf, kvol = 0.0, 0.0
    for ci, cam in enumerate(sc.cams):
        ref = orc.render_bricks(sc.dims, bricks, sc.tf, cam, fr, spacing=sc.spacing)
        # pixels where FP32 may take another discrete decision get no gradient
        ex = (ref["flags"] & (scenes.FLAG["exit"] | scenes.FLAG["ert"] | scenes.FLAG["owner"])) != 0
        g[ci].reshape(-1, 4)[ex] = 0.0
        gi = g[ci].reshape(-1, 4).astype(np.float32).astype(np.float64)
        a, b, amb = orc.grad_bricks(sc.dims, bricks, sc.tf, cam, fr, gi, spacing=sc.spacing, knot_eps=orc.KNOT_EPS)
        rtf = rtf + a
        rvol = rvol + b
        avol = avol + amb
        for eps in (1e-7, -1e-7):
            pa, pb = orc.grad_bricks(sc.dims, bricks, sc.tf, scenes.perturbed_eye(cam, eps), fr, gi, spacing=sc.spacing)
            ktf = np.maximum(ktf, np.abs(pa - a))
            kvol = np.maximum(kvol, np.abs(pb - b))
    dtf, dvol = dev.backward(torch.from_numpy(g.astype(np.float32)).cuda())
    st = dev.stats()
    assert st["samples_backward"] > 0
    l2a, va = scenes.grad_checks(dtf.cpu().numpy(), rtf, "dL/dTF", ktf)
    l2b, vb = scenes.grad_checks(dvol.double().cpu().numpy(), rvol, "dL/dvolume", kvol, avol)
    assert l2a <= 1e-4 and l2b <= 1e-4, (l2a, l2b)
    assert va == 0 and vb == 0, (va, vb)
    dev.release()


def _l2_loss_oracle(orc, sc, bricks, tf, target):
    fr = scenes.oracle_frame(orc, sc)
    loss = 0.0
    for ci, cam in enumerate(sc.cams):
        img = orc.render_bricks(sc.dims, bricks, tf, cam, fr, spacing=sc.spacing)["rgba"]
        loss += np.sum((img - target[ci]) ** 2)
    return loss / (len(sc.cams) * sc.width * sc.height * 4)


def test_tf_gradient_matches_central_differences(orc):
    sc = _scene()
    tf_t = inputs.perturb_tf(sc.tf, seed=0, sigma=0.05)
    bricks = scenes.oracle_bricks(orc, sc)
    fr = scenes.oracle_frame(orc, sc)
    target = [orc.render_bricks(sc.dims, bricks, tf_t, cam, fr, spacing=sc.spacing)["rgba"] for cam in sc.cams]
    # GPU gradient of the same loss through the autograd binding
    dev = scenes.gpu_device(sc, order=False)
    tf = torch.from_numpy(sc.tf).cuda().requires_grad_(True)
    tgt = torch.from_numpy(np.stack(target).reshape(len(sc.cams), sc.height, sc.width, 4)).float().cuda()
    img = dpv.render(dev, tf)
    loss = ((img - tgt) ** 2).mean()
    loss.backward()
    gtf = tf.grad.double().cpu().numpy()
    gmax = np.abs(gtf).max()
    # entries are picked from the oracle's own gradient of the same loss
    N = len(sc.cams) * sc.width * sc.height * 4
    otf = 0.0
    for ci, cam in enumerate(sc.cams):
        img_o = orc.render_bricks(sc.dims, bricks, sc.tf, cam, fr, spacing=sc.spacing)["rgba"]
        a, _ = orc.grad_bricks(sc.dims, bricks, sc.tf, cam, fr, (2.0 / N) * (img_o - target[ci]),
                               spacing=sc.spacing, want_volume=False)
        otf = otf + a
    rng = inputs.rng(0, inputs.STREAM_SELECT)
    nz = np.argwhere(np.abs(otf) > 1e-2 * np.abs(otf).max())
    picks = nz[rng.choice(len(nz), size=min(64, len(nz)), replace=False)]
    eps = 1e-3
    bad = []
    for i, c in picks:
        t1 = sc.tf.copy()
        t1[i, c] += eps
        t0 = sc.tf.copy()
        t0[i, c] -= eps
        h = float(np.float64(t1[i, c]) - np.float64(t0[i, c]))
        fd = (_l2_loss_oracle(orc, sc, bricks, t1, target) - _l2_loss_oracle(orc, sc, bricks, t0, target)) / h
        if abs(fd - gtf[i, c]) > 1e-2 * abs(fd) + 1e-3 * gmax:
            bad.append((int(i), int(c), fd, gtf[i, c]))
    assert not bad, bad
    dev.release()


def test_autograd_matches_direct_backward():
    sc = _scene()
    dev = scenes.gpu_device(sc, order=False)
    tf = torch.from_numpy(sc.tf).cuda().requires_grad_(True)
    vol = torch.from_numpy(sc.field).cuda().requires_grad_(True)
    img = dpv.render(dev, tf, vol)
    w = torch.randn(img.shape, generator=torch.Generator().manual_seed(1)).cuda()
    (img * w).sum().backward()
    dtf, dvol = dev.backward(w)
    # the two backward passes differ only in atomic summation order
    # the same sum both ways (compensated copies, order-free to 1e-9); the
    # autograd gradient is the FP64 table rounded to the TF's float32
    assert torch.allclose(tf.grad.double(), dtf, rtol=2.0 ** -23, atol=1e-9 * float(dtf.abs().max()))
    assert torch.allclose(vol.grad, dvol, rtol=1e-4, atol=1e-6 * float(dvol.abs().max()))
    dev.release()


def test_tf_gradient_cancellation_stress(orc):
    """TF-gradient accumulation under heavy cancellation.  Every sample of
    this scene contributes an exactly representable term, so the FP64
    oracle's sum is exact and any difference is the GPU's accumulation:
    a constant field at s = 63.5 / 256 on a 257-entry table (u = 63.5, both
    lerp weights 1/2), alpha 0 everywhere (T = 1, fragments empty of
    colour, so the only gradient is dL/dalpha of entries 63 and 64, equal
    to dL/dA (1/2) sigma_max dt per sample), dt = 1/64 on a 33^3 grid.  Two
    identical cameras get upstream gradients +4096 + k/16 and -4096 + k'/16
    (seeded k, k' in 0..15): the +-4096 parts cancel between the cameras,
    leaving entries about 10^3 to 10^4 times smaller than the sum of their
    terms' magnitudes.  A plain FP32 running sum loses the remainder to
    rounding; the compensated copies keep it: the GPU entries must equal
    the oracle's to 1e-9 of the largest."""
    dims = (33, 33, 33)
    f = np.full((33, 33, 33), 63.5 / 256, np.float32)
    part = inputs.regular_partition(dims, (2, 2, 2))
    tf = np.zeros((257, 4), np.float32)
    tf[:, :3] = inputs.make_tf(5, n=257)[:, :3]
    cam = scenes.f32_camera(inputs.camera_from_direction(dims, (1.0, 0.7, 0.5)))
    sc = scenes.Scene(f, part, tf, [cam, cam], 64, 64)
    dev = scenes.gpu_device(sc, order=False)
    dev.render()
    g = np.zeros((2, 64, 64, 4), np.float32)
    k = inputs.rng(11, inputs.STREAM_GRAD).integers(0, 16, size=(2, 64, 64))
    g[0, ..., 3] = 4096.0 + k[0] / 16.0
    g[1, ..., 3] = -4096.0 + k[1] / 16.0
    bricks = scenes.oracle_bricks(orc, sc)
    fr = scenes.oracle_frame(orc, sc)
    ref = orc.render_bricks(sc.dims, bricks, tf, cam, fr, spacing=sc.spacing)
    # rays whose sample count FP32 may round differently get no gradient
    ex = (ref["flags"] & scenes.FLAG["exit"]) != 0
    g.reshape(2, -1, 4)[:, ex] = 0.0
    rtf, mag = 0.0, 0.0
    for ci in range(2):
        gi = g[ci].reshape(-1, 4).astype(np.float64)
        rtf = rtf + orc.grad_bricks(sc.dims, bricks, tf, cam, fr, gi, spacing=sc.spacing, want_volume=False)[0]
        mag = mag + orc.grad_bricks(sc.dims, bricks, tf, cam, fr, np.abs(gi), spacing=sc.spacing,
                                    want_volume=False)[0]
    dtf, _ = dev.backward(torch.from_numpy(g).cuda(), volume_grad=False)
    gpu = dtf.cpu().numpy()
    nz = np.argwhere(rtf != 0.0)
    assert sorted(map(tuple, nz.tolist())) == [(63, 3), (64, 3)], nz
    assert np.array_equal(np.argwhere(gpu != 0.0), nz)
    m = np.abs(rtf).max()
    cancel = float(mag[63, 3] / abs(rtf[63, 3]))
    err = float(np.abs(gpu - rtf).max())
    print("cancellation stress: entries %.6e %.6e, sum of |terms| / |entry| %.0f, GPU max abs error %.3e (%.2e of "
          "the largest)" % (rtf[63, 3], rtf[64, 3], cancel, err, err / m))
    assert cancel > 1e3
    assert err <= 1e-9 * m, (gpu[63:65, 3], rtf[63:65, 3])
    dev.release()


def test_autograd_volume_follows_the_tensor():
    """The field handed to the autograd render is the field rendered and
    differentiated: a tensor changed in place after the commit (or another
    tensor) is committed again before the render, so the image and both
    gradients equal those of a device committed from the changed values;
    an unchanged tensor is not committed again; bricks not committed from
    one field cannot be tied to a volume and the render refuses."""
    sc = _scene()
    dev = scenes.gpu_device(sc, order=False)
    vol = torch.from_numpy(sc.field).cuda()
    dev.commit_partition(vol, sc.part, "f32")
    assert not dev.ensure_volume(vol)
    with torch.no_grad():
        vol.mul_(0.7).add_(0.1)                 # in place: the bricks are stale now
    vol.requires_grad_(True)
    tf = torch.from_numpy(sc.tf).cuda().requires_grad_(True)
    img = dpv.render(dev, tf, vol)
    w = torch.randn(img.shape, generator=torch.Generator().manual_seed(4)).cuda()
    (img * w).sum().backward()
    ref = scenes.gpu_device(sc, order=False)
    ref.commit_partition(vol.detach().clone(), sc.part, "f32")
    ref.render()
    assert torch.equal(img.detach(), ref.frames()[0])
    dtf, dvol = ref.backward(w)
    # the same sum both ways (compensated copies, order-free to 1e-9); the
    # autograd gradient is the FP64 table rounded to the TF's float32
    assert torch.allclose(tf.grad.double(), dtf, rtol=2.0 ** -23, atol=1e-9 * float(dtf.abs().max()))
    assert torch.allclose(vol.grad, dvol, rtol=1e-4, atol=1e-6 * float(dvol.abs().max()))
    # the same tensor, unchanged: no new commit
    assert not dev.ensure_volume(vol)
    # bricks committed one by one from a box each: not one known field
    dev.commit_brick(0, sc.part.lo[0], sc.part.hi[0], vol.detach())
    with pytest.raises(ValueError):
        dpv.render(dev, tf, vol)
    dev.release()
    ref.release()


@pytest.mark.parametrize("runs", ["0", "1"])
@pytest.mark.parametrize("split", ["regular", "kd"])
def test_face_buffer_matches_scalar_atomics(monkeypatch, split, runs):
    """The field gradient through the face adjoint buffer (vector atomics per
    cell face, then a gather over every brick storing a node) equals the one
    through scalar atomics into the field, up to atomic summation order; on
    a regular and an uneven k-d partition, ghost copies included; with the
    reductions per sample and per run of samples in one cell."""
    monkeypatch.setenv("DPV_FACE_RUNS", runs)
    dims = (40, 36, 32)
    cams = inputs.sphere_cameras(dims, 2, seed=4)
    kw = dict(splits=(2, 2, 2)) if split == "regular" else dict(kd=7)
    sc = scenes.make(dims, nblobs=10, cams=cams, width=48, height=40, **kw)
    dev = scenes.gpu_device(sc, order=False)
    dev.render()
    g = torch.from_numpy(inputs.rng(0, inputs.STREAM_GRAD).normal(size=(len(sc.cams), sc.height, sc.width, 4))
                         .astype(np.float32)).cuda()
    monkeypatch.delenv("DPV_FACE_GRAD", raising=False)
    dev.reset_stats()
    dtf1, dvol1 = dev.backward(g)
    l1 = dev.stats()["kernel_launches"]
    monkeypatch.setenv("DPV_FACE_GRAD", "0")
    dev.reset_stats()
    dtf0, dvol0 = dev.backward(g)
    l0 = dev.stats()["kernel_launches"]
    assert l1 == l0 + 1                      # the gather ran on the face path only
    assert float(dvol0.abs().max()) > 0
    assert torch.allclose(dvol1, dvol0, rtol=1e-5, atol=1e-6 * float(dvol0.abs().max()))
    # TF entries: the same terms on both paths, summed in another atomic
    # order by compensated copies: equal to 1e-9 of the largest entry
    assert torch.allclose(dtf1, dtf0, rtol=0, atol=1e-9 * float(dtf0.abs().max()))
    dev.release()


@pytest.mark.parametrize("split", ["regular", "kd"])
def test_face_buffer_in_brick_groups(monkeypatch, split):
    """Where the face buffer does not fit, the adjoint takes the bricks in
    groups: it replays one group's items into the buffer, gathers the
    group's slots and adds them into the field, then takes the next group.
    Forced here with at most n bricks per group: the field and TF gradients
    equal the one-buffer pass up to atomic summation order, and each extra
    group costs one replay and one gather launch."""
    dims = (40, 36, 32)
    cams = inputs.sphere_cameras(dims, 2, seed=4)
    kw = dict(splits=(2, 2, 2)) if split == "regular" else dict(kd=7)
    sc = scenes.make(dims, nblobs=10, cams=cams, width=48, height=40, **kw)
    K = sc.part.num_ranks
    dev = scenes.gpu_device(sc, order=False)
    dev.render()
    g = torch.from_numpy(inputs.rng(2, inputs.STREAM_GRAD).normal(size=(len(sc.cams), sc.height, sc.width, 4))
                         .astype(np.float32)).cuda()
    monkeypatch.delenv("DPV_FACE_GRAD", raising=False)
    monkeypatch.delenv("DPV_FACE_GROUP", raising=False)
    dev.reset_stats()
    dtf0, dvol0 = dev.backward(g)
    l0 = dev.stats()["kernel_launches"]
    assert float(dvol0.abs().max()) > 0
    for n in (1, 3):
        monkeypatch.setenv("DPV_FACE_GROUP", str(n))
        dev.reset_stats()
        dtf, dvol = dev.backward(g)
        groups = -(-K // n)
        assert dev.stats()["kernel_launches"] == l0 + 2 * (groups - 1)
        assert torch.allclose(dvol, dvol0, rtol=1e-5, atol=1e-6 * float(dvol0.abs().max()))
        assert torch.allclose(dtf, dtf0, rtol=0, atol=1e-9 * float(dtf0.abs().max()))
    dev.release()


@pytest.mark.parametrize("split", ["regular", "kd"])
def test_adjoint_overwrites_every_output(monkeypatch, split):
    """dpvBackward overwrites its outputs: caller buffers filled with NaN
    come back finite, equal to the one-buffer pass, whether the face buffer
    holds every brick or the bricks go in groups (where the first group to
    reach a node stores it and later groups add: no node may be missed, on
    the owned boxes' surfaces least of all), and on the scalar-atomic
    path."""
    dims = (40, 36, 32)
    cams = inputs.sphere_cameras(dims, 2, seed=5)
    kw = dict(splits=(2, 2, 2)) if split == "regular" else dict(kd=7)
    sc = scenes.make(dims, nblobs=10, cams=cams, width=48, height=40, **kw)
    dev = scenes.gpu_device(sc, order=False)
    dev.render()
    g = torch.from_numpy(inputs.rng(3, inputs.STREAM_GRAD).normal(size=(len(sc.cams), sc.height, sc.width, 4))
                         .astype(np.float32)).cuda()
    lib = dpv.load()

    def run():
        dtf = torch.full((dev.ntf, 4), float("nan"), dtype=torch.float64, device="cuda")
        dvol = torch.full((dims[2], dims[1], dims[0]), float("nan"), dtype=torch.float32, device="cuda")
        assert lib.dpvBackward(dev._h, g.data_ptr(), dtf.data_ptr(), dvol.data_ptr()) == 0
        torch.cuda.synchronize()
        assert bool(torch.isfinite(dtf).all()) and bool(torch.isfinite(dvol).all())
        return dtf, dvol

    monkeypatch.delenv("DPV_FACE_GRAD", raising=False)
    monkeypatch.delenv("DPV_FACE_GROUP", raising=False)
    dtf0, dvol0 = run()
    assert float(dvol0.abs().max()) > 0
    for env in (("DPV_FACE_GROUP", "1"), ("DPV_FACE_GROUP", "3"), ("DPV_FACE_GRAD", "0")):
        monkeypatch.setenv(*env)
        dtf, dvol = run()
        monkeypatch.delenv(env[0])
        assert torch.allclose(dvol, dvol0, rtol=1e-5, atol=1e-6 * float(dvol0.abs().max())), env
        assert torch.allclose(dtf, dtf0, rtol=0, atol=1e-9 * float(dtf0.abs().max())), env
    dev.release()


def test_adjoint_run_to_run_spread():
    """The forward has no atomics and is bit-deterministic (test_gpu_parity);
    the adjoint sums with atomics in whatever order the hardware takes, so
    two runs on the same inputs differ by rounding.  Reported and bounded:
    relative L2 and max over entries above 1e-3 of the largest, below 1e-5
    for the field gradient (FP32 atomics) and below 1e-9 for the TF gradient
    (compensated copies, then FP64)."""
    sc = _scene()
    dev = scenes.gpu_device(sc, order=False)
    dev.render()
    g = torch.from_numpy(inputs.rng(3, inputs.STREAM_GRAD).normal(size=(len(sc.cams), sc.height, sc.width, 4))
                         .astype(np.float32)).cuda()
    runs = [tuple(t.double().cpu().numpy() for t in dev.backward(g)) for _ in range(4)]
    for name, idx in (("dL/dTF", 0), ("dL/dvolume", 1)):
        ref = runs[0][idx]
        big = np.abs(ref) > 1e-3 * np.abs(ref).max()
        l2 = max(np.linalg.norm(r[idx] - ref) / np.linalg.norm(ref) for r in runs[1:])
        mx = max(float((np.abs(r[idx] - ref)[big] / np.abs(ref[big])).max()) for r in runs[1:])
        print("%s run-to-run: rel L2 %.2e, max rel %.2e" % (name, l2, mx))
        bar = 1e-9 if idx == 0 else 1e-5
        assert l2 <= bar and mx <= bar
    dev.release()
