"""GPU parity with a transfer-function domain other than [0, 1].

The field is stretched past both ends of the domain, so samples take the
clamped first and last entries and the clamp zeroes du/ds on both sides.
Forward frames against the FP64 oracle at 1e-5 per channel on the pixels
it does not flag; TF and field gradients against the oracle's reverse-mode
gradient at the gradient bar of scenes.grad_checks (the oracle's knot
ambiguity covers samples within rounding of vmin or vmax whose corners
reach past it)."""
import numpy as np
import pytest
import torch

from paper_2407_00179_b300 import build, dpv, inputs

import scenes

pytestmark = pytest.mark.gpu

TOL = 1e-5
DOMAINS = [(0.2, 0.8), (-0.25, 1.6)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    dpv.load()


def _scene(domain, storage="f32", ert=0.0, ncam=2):
    dims = (40, 36, 32)
    cams = inputs.sphere_cameras(dims, ncam, seed=4)
    sc = scenes.make(dims, splits=(2, 2, 2), nblobs=10, cams=cams, width=48, height=40, ert=ert, storage=storage)
    vmin, vmax = domain
    w = vmax - vmin
    f = sc.field.astype(np.float64)
    f = np.cbrt((f - f.min()) / (f.max() - f.min()))      # about 15 % of the nodes on each clamped side
    sc.field = (vmin - 0.5 * w + 2.0 * w * f).astype(np.float32)
    return sc


def _device(sc, domain):
    dev = scenes.gpu_device(sc, order=True)
    dev.set_tf(torch.from_numpy(sc.tf).cuda(), *domain)
    return dev


def _sides(sc, domain):
    """Fractions of the field's nodes below, inside and above the domain."""
    f = sc.field
    return np.array([(f < domain[0]).mean(), ((f >= domain[0]) & (f <= domain[1])).mean(), (f > domain[1]).mean()])


@pytest.mark.parametrize("storage", ["f32", "f16"])
@pytest.mark.parametrize("domain", DOMAINS)
def test_forward_non_unit_domain(orc, domain, storage):
    sc = _scene(domain, storage=storage)
    assert _sides(sc, domain).min() > 0.1
    dev = _device(sc, domain)
    dev.render()
    bricks = scenes.oracle_bricks(orc, sc)
    fr = scenes.oracle_frame(orc, sc)
    for ci, cam in enumerate(sc.cams):
        ref = orc.render_bricks(sc.dims, bricks, sc.tf, cam, fr, spacing=sc.spacing, vmin=domain[0], vmax=domain[1])
        img = dev.map_frame(ci)[0].double().cpu().numpy().reshape(-1, 4)
        ex = (ref["flags"] & (scenes.FLAG["exit"] | scenes.FLAG["owner"])) != 0
        assert ex.mean() < 0.05
        err = np.abs(img - ref["rgba"])[~ex]
        print("domain %s %s camera %d: max abs %.2e over %d pixels" % (domain, storage, ci, err.max(), (~ex).sum()))
        assert err.max() <= TOL
        order = dev.order(ci).reshape(-1, sc.part.num_ranks).cpu().numpy()
        assert np.array_equal(order[~ex], ref["order"][~ex])
        # the same frame with the unit domain differs: the domain is used
        ref01 = orc.render_bricks(sc.dims, bricks, sc.tf, cam, fr, spacing=sc.spacing)
        assert np.abs(img - ref01["rgba"])[~ex].max() > 1e-2
    dev.release()


@pytest.mark.parametrize("domain", DOMAINS)
def test_gradients_non_unit_domain(orc, domain):
    sc = _scene(domain)
    dev = _device(sc, domain)
    dev.render()
    g = inputs.rng(7, inputs.STREAM_GRAD).normal(size=(len(sc.cams), sc.height, sc.width, 4))
    bricks = scenes.oracle_bricks(orc, sc)
    fr = scenes.oracle_frame(orc, sc)
    kw = dict(spacing=sc.spacing, vmin=domain[0], vmax=domain[1])
    rtf, rvol, avol, ktf, kvol = 0.0, 0.0, 0.0, 0.0, 0.0
    for ci, cam in enumerate(sc.cams):
        ref = orc.render_bricks(sc.dims, bricks, sc.tf, cam, fr, **kw)
        ex = (ref["flags"] & (scenes.FLAG["exit"] | scenes.FLAG["ert"] | scenes.FLAG["owner"])) != 0
        g[ci].reshape(-1, 4)[ex] = 0.0
        gi = g[ci].reshape(-1, 4).astype(np.float32).astype(np.float64)
        a, b, amb = orc.grad_bricks(sc.dims, bricks, sc.tf, cam, fr, gi, knot_eps=orc.KNOT_EPS, **kw)
        rtf, rvol, avol = rtf + a, rvol + b, avol + amb
        for eps in (1e-7, -1e-7):
            pa, pb = orc.grad_bricks(sc.dims, bricks, sc.tf, scenes.perturbed_eye(cam, eps), fr, gi, **kw)
            ktf = np.maximum(ktf, np.abs(pa - a))
            kvol = np.maximum(kvol, np.abs(pb - b))
    # both end entries collect the clamped samples
    n = sc.tf.shape[0]
    assert np.abs(rtf[0]).max() > 1e-3 * np.abs(rtf).max() and np.abs(rtf[n - 1]).max() > 1e-3 * np.abs(rtf).max()
    dtf, dvol = dev.backward(torch.from_numpy(g.astype(np.float32)).cuda())
    gtf, gvol = dtf.cpu().numpy(), dvol.double().cpu().numpy()
    l2a, va = scenes.grad_checks(gtf, rtf, "dL/dTF", ktf)
    l2b, vb = scenes.grad_checks(gvol, rvol, "dL/dvolume", kvol, avol)
    assert l2a <= 1e-4 and l2b <= 1e-4, (l2a, l2b)
    assert va == 0 and vb == 0, (va, vb)
    # nodes whose every neighbour lies outside the domain on one side get no
    # gradient on either path
    f = sc.field
    pad = np.pad(f, 1, mode="edge")
    nbmax = np.max([pad[1 + dz:1 + dz + f.shape[0], 1 + dy:1 + dy + f.shape[1], 1 + dx:1 + dx + f.shape[2]]
                    for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)], axis=0)
    nbmin = np.min([pad[1 + dz:1 + dz + f.shape[0], 1 + dy:1 + dy + f.shape[1], 1 + dx:1 + dx + f.shape[2]]
                    for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)], axis=0)
    out = (nbmax < domain[0]) | (nbmin > domain[1])
    assert out.sum() > 100
    assert np.all(rvol[out] == 0.0) and np.all(gvol[out] == 0.0)
    dev.release()
