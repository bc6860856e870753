"""Seeded scenes used by the parity tests: the same inputs go to the CUDA
path (through the C ABI) and to the FP64 oracle."""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np
import torch

from paper_2407_00179_b300 import inputs

FLAG = {"hit": 1, "exit": 2, "owner": 4, "ert": 8}


@dataclass
class Scene:
    field: np.ndarray            # (nz, ny, nx) float32
    part: inputs.Partition
    tf: np.ndarray               # (n, 4) float32
    cams: List[inputs.Camera]
    width: int
    height: int
    step: float = 0.5
    sigma_max: float = 8.0
    ert: float = 0.0
    storage: str = "f32"
    tile: tuple = (0, 0)
    staged: bool = False

    @property
    def dims(self):
        return (self.field.shape[2], self.field.shape[1], self.field.shape[0])

    @property
    def spacing(self):
        """Node spacing exactly as the C ABI receives it (float32)."""
        return float(np.float32(1.0 / (max(self.dims) - 1)))


def f32_camera(c: inputs.Camera) -> inputs.Camera:
    """The camera exactly as the C ABI receives it (float32 fields), so the
    oracle and the GPU see the same rays."""
    r = lambda v: tuple(float(x) for x in np.asarray(v, np.float32))
    return inputs.Camera(r(c.eye), r(c.center), r(c.up), float(np.float32(c.fovy_deg)))


def small(seed=0, width=256, height=256, storage="f32", ert=0.0, tile=(0, 0)) -> Scene:
    """64^3 sum of 8 blobs, 2x1x1 bricks, one camera from (1, 0.7, 0.5)."""
    dims = (64, 64, 64)
    f = inputs.field_small(seed, dims).numpy()
    return Scene(f, inputs.regular_partition(dims, (2, 1, 1)), inputs.make_tf(1234),
                 [f32_camera(inputs.camera_from_direction(dims, (1.0, 0.7, 0.5)))], width, height, storage=storage,
                 ert=ert,
                 tile=tile)


def make(dims, splits=None, kd=None, nblobs=8, seed=0, cams=None, width=64, height=48, **kw) -> Scene:
    f = inputs.blob_field(dims, inputs.blob_params(nblobs, dims, seed)).numpy()
    part = inputs.kd_partition(dims, kd, seed=seed) if kd else inputs.regular_partition(dims, splits or (1, 1, 1))
    cams = cams if cams is not None else [inputs.camera_from_direction(dims, (1.0, 0.7, 0.5))]
    return Scene(f, part, inputs.make_tf(1234), [f32_camera(c) for c in cams], width, height, **kw)


def gpu_device(sc: Scene, order=True):
    from paper_2407_00179_b300 import dpv
    dev = dpv.Device(sc.part.num_ranks)
    dev.set_geometry(sc.dims)
    fld = torch.from_numpy(sc.field).cuda()
    dev.commit_partition(fld, sc.part, sc.storage)
    dev.set_tf(torch.from_numpy(sc.tf).cuda())
    dev.set_cameras(sc.cams)
    dev.set_frame(sc.width, sc.height, step_voxels=sc.step, sigma_max=sc.sigma_max, ert=sc.ert, tile=sc.tile,
                  order=order, staged=sc.staged)
    return dev


def oracle_bricks(orc, sc: Scene):
    return orc.make_bricks(sc.field, sc.part, orc.DTYPE_NAMES[sc.storage])


def oracle_frame(orc, sc: Scene):
    return orc.Frame(sc.width, sc.height, step_voxels=sc.step, sigma_max=sc.sigma_max, ert=sc.ert)


def o_bricks(orc, sc: Scene, cam, **kw):
    """Oracle partitioned render of camera `cam` with the scene's inputs."""
    return orc.render_bricks(sc.dims, oracle_bricks(orc, sc), sc.tf, cam, oracle_frame(orc, sc), spacing=sc.spacing,
                             **kw)


def o_full(orc, sc: Scene, cam, field=None, **kw):
    f = sc.field if field is None else field
    return orc.render_full(f, sc.tf, cam, oracle_frame(orc, sc), spacing=sc.spacing, **kw)


def grad_checks(gpu, ref, what, kappa=None, amb=None):
    """Gradient bar: relative L2 <= 1e-4, and on entries above 1e-3 of
    the largest, |gpu - ref| <= 1e-3 |ref| + 2 kappa + amb.

    kappa is how much the FP64 oracle's own answer moves when the eye is
    perturbed by 1e-7 relative (about one FP32 rounding of the ray
    geometry).  Entries that are sums of large cancelling terms are only
    determined to that level once the geometry is rounded to FP32, whatever
    the arithmetic after it.  Measured over every gradient test: at most 3
    entries of a test need the allowance at all, and the largest needs
    1.01 kappa beyond 1e-3 |ref| + amb; 2 kappa keeps a margin of two.

    amb is the oracle's knot ambiguity of a field gradient: where a sample
    lies within rounding of a TF knot whose slope changes, either one-sided
    derivative is correct, and amb is how far that can move the entry.  The
    relative L2 is taken over what is left of each entry's error after amb."""
    m = np.abs(ref).max()
    assert m > 0
    big = np.abs(ref) > 1e-3 * m
    err = np.abs(gpu - ref)
    rel = err[big] / np.abs(ref[big])
    a = np.zeros_like(ref) if amb is None else amb
    l2 = np.linalg.norm(np.maximum(err - a, 0.0)) / np.linalg.norm(ref)
    k = np.zeros_like(ref) if kappa is None else kappa
    bound = 1e-3 * np.abs(ref) + 2.0 * k + a
    viol = big & (err > bound)
    # entries that need the kappa allowance: beyond 1e-3 |ref| + amb, within
    # the full bound; and the distribution of |gpu - ref| / kappa over them
    need = big & (err > 1e-3 * np.abs(ref) + a) & ~viol
    if need.any():
        r = (err[need] - 1e-3 * np.abs(ref[need]) - a[need]) / np.maximum(k[need], 1e-300)
        print("%s: %d of %d entries use the kappa allowance; (|gpu - ref| - 1e-3|ref| - amb) / kappa: "
              "median %.2f, 90th pct %.2f, max %.2f" % (what, need.sum(), big.sum(), np.median(r),
                                                         np.percentile(r, 90), r.max()))
    else:
        print("%s: no entry uses the kappa allowance" % what)
    w = np.argsort(rel)[-3:]
    print("%s: max rel %.2e (over %d entries), rel L2 %.2e (raw %.2e), %d beyond 1e-3|ref| + 2 kappa + amb "
          "(%d entries with amb > 0); worst: %s" % (
              what, rel.max(), big.sum(), l2, np.linalg.norm(gpu - ref) / np.linalg.norm(ref), viol.sum(),
              int((a > 0).sum()),
              ", ".join("gpu %.6e ref %.6e kappa %.1e amb %.1e (|ref|/max %.1e)" % (
                  gpu[big][i], ref[big][i], k[big][i], a[big][i], abs(ref[big][i]) / m) for i in w)))
    for i in np.flatnonzero(viol.reshape(-1))[:4]:
        print("  beyond: index %d gpu %.6e ref %.6e bound %.2e (kappa %.1e, |ref|/max %.1e)" % (
            i, gpu.reshape(-1)[i], ref.reshape(-1)[i], bound.reshape(-1)[i], k.reshape(-1)[i],
            abs(ref.reshape(-1)[i]) / m))
    return l2, int(viol.sum())


def perturbed_eye(cam, eps):
    """The camera with its eye scaled by (1 + eps): about one FP32 rounding
    of the ray geometry for eps = 1e-7."""
    return inputs.Camera(tuple(float(x) * (1.0 + eps) for x in cam.eye), cam.center, cam.up, cam.fovy_deg)
